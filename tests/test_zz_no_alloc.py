"""ic_apply_static: the preconditioner application that allocates nothing.

Some callers cannot allocate GPU memory where they apply the preconditioner: a plugin
inside another framework that owns the device's memory budget and gives it no
allocator, or a loop with a hard latency limit where a cudaMalloc (which may
synchronise the device) is not allowed.  They use this entry point; its scratch is a
static device array of the library.  Checked here through the C ABI against ic_apply
on the same factor and against the CPU oracle's application, on two calls in a row
(the second call reuses the scratch the first one left behind), with the timeout
record read back clear.  This file is collected last so that a run stopping at the
first failure has run every other test.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ick():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1601_05871_gb300.build import build
    build()
    import paper_1601_05871_gb300 as m
    m.load()
    return m


def test_apply_static_matches_apply_and_oracle_twice(ick, orc):
    import torch
    prob = synth.laplace3d_27pt(20)
    perm, ranges = ick.ic_nd_grid(20, 20, 20, 1, 1000)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 2, perm, ranges, block_rows=1000)
    ick.ic_numeric(h, torch.from_numpy(prob.vals).cuda())
    o = orc.OracleIC.from_problem(prob, perm, 2)
    assert o.numeric(prob.vals) == 0
    g = np.random.default_rng(9)
    for call in range(2):
        rh = g.standard_normal(prob.n)
        r = torch.from_numpy(rh).cuda()
        z_ref = torch.empty_like(r)
        z_st = torch.full_like(r, float("nan"))
        ick.ic_apply(h, r, z_ref)
        ick.ic_apply_static(h, r, z_st)
        ick.ic_apply_static_status()
        ick.ic_apply_status(h)
        a, b = z_ref.cpu().numpy(), z_st.cpu().numpy()
        zo = o.apply(rh)
        assert np.all(np.isfinite(b)), call
        # the tolerance of the other solve tests: 1e-11 relative to the largest entry
        assert np.abs(a - b).max() <= 1e-11 * np.abs(a).max(), call
        assert np.abs(b - zo).max() <= 1e-11 * np.abs(zo).max(), call


def test_apply_static_rejects_aliasing_and_too_many_rows(ick):
    import torch
    prob = synth.poisson2d_5pt(16, 16)
    h = ick.ic_symbolic(prob.rowptr, prob.colind, 1)
    ick.ic_numeric(h, torch.from_numpy(prob.vals).cuda())
    v = torch.zeros(prob.n, dtype=torch.float64, device="cuda")
    with pytest.raises(ick.IckError) as e:
        ick.ic_apply_static(h, v, v)
    assert e.value.status == ick.ick.IC_ERR_ARG
    big = synth.diffusion3d_7pt(103, sigma=0.5, seed=1)  # 1,092,727 rows > 2^20
    hb = ick.ic_symbolic(big.rowptr, big.colind, 0, block_rows=8192)
    ick.ic_numeric(hb, torch.from_numpy(big.vals).cuda())
    x = torch.zeros(big.n, dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(ick.IckError) as e:
        ick.ic_apply_static(hb, x, y)
    assert e.value.status == ick.ick.IC_ERR_ARG and "1048576" in str(e.value)
