"""The seeded input recipes stated in the design notes, checked on the
generators themselves (sizes, coefficient structure, seeds): the benchmark
problem's n, nnz, subdomain sizes and channel contrast; the first
configuration's stencil; the batch generator's size rule.  No arithmetic of
the method is involved."""

import numpy as np
import scipy.sparse as sp

import awg_inputs as gi
import oracle as O


def test_config2_recipe():
    p = gi.config2()
    assert p.n == 512 * 512 and p.rowptr[-1] == 1_308_672
    assert p.nparts == 256 and p.overlap == 2 and p.tau == 0.1
    A = O.csr_from(p.rowptr, p.colidx, p.val, p.n)
    assert abs(A - A.T).max() == 0
    subs = O.grow_subdomains(A, p.part, p.nparts, p.overlap)
    sizes = np.array([len(s) for s in subs])
    assert sizes.sum() == 324_484 and sizes.max() == 1284
    # harmonic-mean faces of kappa in {1, 1e6}: off-diagonals -1, -1e6 or the
    # mean across a channel edge 2e6/(1e6 + 1); nothing else
    off = -A.data[A.indices != np.repeat(np.arange(p.n), np.diff(A.indptr))]
    vals = np.unique(np.round(off, 6))
    assert set(vals.tolist()) <= {1.0, 1e6, round(2e6 / (1e6 + 1), 6)}
    assert np.array_equal(p.b, np.random.default_rng(0).standard_normal(p.n))


def test_config1_recipe():
    p = gi.config1()
    assert p.n == 4096 and p.rowptr[-1] == 20_224 and p.nparts == 16 and p.overlap == 1
    A = O.csr_from(p.rowptr, p.colidx, p.val, p.n)
    assert np.all(A.diagonal() == 4.0)
    off = (A - sp.diags(A.diagonal())).tocsr()
    off.eliminate_zeros()
    assert set(np.unique(off.data).tolist()) == {-1.0}


def test_batch_recipe():
    probs = gi.batch_channels(4, Lmin=128, Lmax=256)
    for j, q in enumerate(probs):
        L = int(round(np.sqrt(q.n)))
        assert L * L == q.n and 128 <= L <= 256
        qq = 8 + int(round(16 * (L - 128) / 640))
        assert q.nparts == qq * qq
