"""lbm_reduce_static, the reduction that allocates nothing, against lbm_reduce.

Callers that may not allocate device memory when they need a conservation check (an
application whose device memory all belongs to its own pool, or a latency-critical
loop that cannot absorb the device-wide synchronisation of cudaMalloc) use
lbm_reduce_static on a population array they already hold.  This file checks, through
the C ABI, that two calls in a row give what the allocating lbm_reduce gives for the
same state.  It is named to be collected last and also passes alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _state(lbm, precision):
    from paper_2405_12082_gb300 import workloads as Wk
    import torch
    grid = lbm.make_grid(28, 28, 12, 12.0, precision=precision, wall="halfway")
    force = lbm.make_force(g=(0.0, 0.0, 2e-5),
                           trigger=Wk.trigger_dict(h=2e-5, R=12.0, nz=12, period=30.0,
                                                   modes=[(1, 0.5, 0.0), (2, 0.5, 0.7)], t_end=100))
    L = lbm.Lattice(grid, lbm.lbm_relax(1.6), force)
    L.init("laminar", noise_amp=2e-3, seed=Wk.SEED)
    L.step(6)                                       # even t: natural layout
    info = L.info()
    raw = torch.empty(info["population_bytes"], dtype=torch.uint8, device="cuda")
    lbm.lbm_get_raw(L.ctx, raw, info["population_bytes"])
    return L, raw


@pytest.mark.parametrize("precision", ["f32", "f64", "f16s"])
def test_static_reduce_matches_reduce_twice(lbm_lib, precision):
    import torch
    lbm = lbm_lib
    L, raw = _state(lbm, precision)
    expect = np.array(lbm.lbm_reduce(L.ctx))
    esize = {"f64": 8, "f32": 4, "f16s": 2}[precision]
    n_cells = raw.numel() // (27 * esize)
    out = torch.full((5,), float("nan"), dtype=torch.float64, device="cuda")
    scale = max(np.max(np.abs(expect[:4])), 1e-300)
    for _ in range(2):
        out.fill_(float("nan"))
        lbm.lbm_reduce_static(raw, precision, 0, n_cells, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        # same sums in a different order: FP64 rounding only
        assert np.max(np.abs(got[:4] - expect[:4])) <= 1e-12 * scale + 1e-15, (got, expect)
        assert got[4] == expect[4] == 0
    L.close()


def test_static_reduce_rejects_bad_sizes(lbm_lib):
    import torch
    lbm = lbm_lib
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    buf = torch.zeros(27 * 4, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_reduce_static(buf, "f32", 0, lbm.LBM_STATIC_REDUCE_MAX_CELLS + 1, out)
    assert ei.value.status == lbm.LBM_EINVAL
    with pytest.raises(lbm.LbmError):
        lbm.lbm_reduce_static(buf, "f32", 0, 0, out)
    with pytest.raises(lbm.LbmError):            # the output must be device memory
        lbm.lbm_reduce_static(buf, "f32", 0, 4, np.zeros(5))
