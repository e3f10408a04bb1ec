"""Host logic of the two-slab decomposition (no GPU): every global row is owned by exactly
one slab, the cut plane is stored on both sides, split/join round-trip."""
import pytest
import torch

from paper_2609_16424_b300.partition import slab_maps


@pytest.mark.parametrize("dim,n,k,cut", [(2, (5, 4), 2, 1), (2, (3, 6), 3, 4), (3, (2, 3, 4), 2, 2),
                                         (3, (3, 2, 5), 1, 1), (3, (2, 2, 3), 4, 2)])
def test_slab_maps(dim, n, k, cut):
    n_g, rows, owned = slab_maps(dim, n, k, cut)
    nv_g = 1
    for c in range(dim):
        nv_g *= k * n[c] + 1
    ne_g = 1
    for c in range(dim):
        ne_g *= n[c]
    assert n_g == 2 * dim * nv_g + ne_g * k ** dim
    count = torch.zeros(n_g, dtype=torch.long)
    seen = torch.zeros(n_g, dtype=torch.long)
    for r, o in zip(rows, owned):
        assert r.min() >= 0 and r.max() < n_g and len(torch.unique(r)) == len(r)
        count[r[o]] += 1
        seen[r] += 1
    assert torch.all(count == 1)
    plane = nv_g // (k * n[-1] + 1)
    dup = seen == 2
    assert dup.sum() == 2 * dim * plane                    # x and v rows of the cut plane
    # round trip of a global vector
    v = torch.arange(n_g, dtype=torch.float64)
    parts = [v[r] for r in rows]
    out = torch.empty_like(v)
    for r, o, x in zip(rows, owned, parts):
        out[r[o]] = x[o]
    assert torch.equal(out, v)
