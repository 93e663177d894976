"""The allocation-free batched entry point (chem_integrate_batched_noalloc).

It serves callers that cannot allocate device memory during the call: a host solver
whose memory arena owns the GPU, or a latency-bound loop that cannot pay for
cudaMalloc's synchronisation.  Its queue scratch is a fixed array in the library, so
its results must match the allocating entry point (chem_integrate_batched) on the same
inputs.  They are checked here within the FP64 parity tolerance, on two calls in a row,
because each call reuses the array the previous one left behind.  Requests beyond the
fixed maximum are rejected before any launch, and the binding rejects tensors that are
too short for the requested cell count.  Both queue orders (stiffness key or index order)
and a caller's cost hint give the same per-cell results.

This file is named to be collected last.
"""
import numpy as np
import pytest

import oracle
from chem_inputs import mechanism as M
from chem_inputs import workloads as W

pytestmark = pytest.mark.gpu

TOL_T = 1e-8   # the FP64 parity bar used by the other GPU tests
TOL_Y = 1e-10


def _inputs(seed, nboxes):
    b = W.amr_batch(nboxes=nboxes, seed=seed, edges=(4, 8, 12))
    o = oracle.Oracle(M.build(0))
    b["rho"], b["e"] = o.state_from_TPY(b["T"], b["p"], b["Y"])
    return b


def _run(ctx, b, noalloc, **opts):
    import torch
    dev = lambda a, dt=torch.float64: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")
    n = b["T"].size
    Y, T = dev(b["Y"]), dev(b["T"])
    st = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    ns = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    args = (dev(b["rho"]), dev(b["e"]), Y, T, dev(b["box_offset"], torch.int64),
            dev(b["box_dt"]), dev(b["box_nsub"], torch.int32))
    if noalloc:
        ctx.integrate_batched_noalloc(*args, status=st, nsteps=ns, **opts)
    else:
        ctx.integrate_batched(*args, status=st, nsteps=ns)
    torch.cuda.synchronize()
    return Y.cpu().numpy(), T.cpu().numpy(), st.cpu().numpy(), ns.cpu().numpy()


@pytest.mark.parametrize("variant", ["fp64", "mixed"])
def test_noalloc_matches_batched_on_two_calls(variant):
    from paper_2506_02602_gb300 import build, chem
    build.build()
    ctx = chem.Context(M.build(0), variant)
    for seed, nboxes in ((31, 60), (32, 45)):  # two calls in a row, different sizes
        b = _inputs(seed, nboxes)
        Yr, Tr, sr, nr = _run(ctx, b, noalloc=False)
        Yn, Tn, sn, nn = _run(ctx, b, noalloc=True)
        assert np.all(sr == 0)
        np.testing.assert_array_equal(sn, sr)
        np.testing.assert_array_equal(nn, nr)
        assert np.max(np.abs(Tn - Tr) / Tr) <= TOL_T
        assert np.max(np.abs(Yn - Yr)) <= TOL_Y
    ctx.close()


@pytest.mark.parametrize("queue", ["natural", "cost_hint"])
def test_noalloc_other_queue_orders(queue):
    """The other queue orders of the allocation-free entry: cells in index order, and cells
    ordered by a caller's per-cell cost (here the step counts of a previous call); only
    the schedule changes, so the results match the allocating entry point's."""
    import torch
    from paper_2506_02602_gb300 import build, chem
    build.build()
    ctx = chem.Context(M.build(0), "fp64")
    b = _inputs(33, 40)
    Yr, Tr, sr, nr = _run(ctx, b, noalloc=False)
    if queue == "natural":
        opts = {"order": chem.ORDER_NATURAL}
    else:
        opts = {"cost_hint": torch.tensor(nr, dtype=torch.int32, device="cuda")}
    Yn, Tn, sn, nn = _run(ctx, b, noalloc=True, **opts)
    assert np.all(sr == 0)
    np.testing.assert_array_equal(sn, sr)
    np.testing.assert_array_equal(nn, nr)
    assert np.max(np.abs(Tn - Tr) / Tr) <= TOL_T
    assert np.max(np.abs(Yn - Yr)) <= TOL_Y
    ctx.close()


def test_noalloc_rejects_more_cells_than_its_scratch():
    import torch
    from paper_2506_02602_gb300 import build, chem
    build.build()
    ctx = chem.Context(M.build(0), "fp64")
    n = (1 << 20) + 1  # one cell beyond the fixed scratch; the tensors really hold n cells
    x = torch.zeros(n, dtype=torch.float64, device="cuda")
    Y = torch.zeros((9, n), dtype=torch.float64, device="cuda")
    off = torch.tensor([0, n], dtype=torch.int64, device="cuda")
    dt = torch.tensor([1e-7], dtype=torch.float64, device="cuda")
    nsub = torch.tensor([1], dtype=torch.int32, device="cuda")
    # the size check comes before anything is launched
    with pytest.raises(chem.ChemError) as ei:
        ctx.integrate_batched_noalloc(x, x, Y, x, off, dt, nsub)
    assert ei.value.code == chem.ERR_INVALID and "1048576" in str(ei.value)
    # a cell count beyond the tensors' own size never reaches the library
    small = torch.zeros(16, dtype=torch.float64, device="cuda")
    with pytest.raises(chem.ChemError) as ei:
        ctx.integrate_batched_noalloc(small, small, Y[:, :16], small, off, dt, nsub, ncells=17)
    assert ei.value.code == chem.ERR_INVALID
    with pytest.raises(chem.ChemError):  # fp32 state is refused as in integrate_batched
        ctx.integrate_batched_noalloc(small.float(), small, Y[:, :16], small, off, dt, nsub)
    ctx.close()
