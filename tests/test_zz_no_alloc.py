"""lbm_reduce_static, the reduction that allocates nothing, against lbm_reduce.

Callers that may not allocate device memory when they need a conservation check (an
application whose device memory all belongs to its own pool, or a latency-critical
loop that cannot absorb the device-wide synchronisation of cudaMalloc) use
lbm_reduce_static on a population array they already hold.  This file checks, through
the C ABI, that two calls in a row give what the allocating lbm_reduce gives for the
same state, in every storage precision, that a non-finite value is counted, and that
bad arguments are refused before any launch.  It is named to be collected last and
also passes alone in a fresh process.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

ESIZE = {"f64": 8, "f32": 4, "f16s": 2, "bf16": 2}


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


@pytest.mark.parametrize("precision", ["f32", "f64", "f16s", "bf16"])
def test_static_reduce_matches_reduce_twice(lbm_lib, precision):
    import torch
    lbm = lbm_lib
    L, raw = _state(lbm, precision)
    expect = np.array(lbm.lbm_reduce(L.ctx))
    n_cells = raw.numel() // (27 * ESIZE[precision])
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


@pytest.mark.parametrize("precision", ["f32", "bf16"])
def test_static_reduce_counts_a_non_finite_cell(lbm_lib, precision):
    """A NaN written into the host copy of the raw state (one population of one cell)
    is counted once: out[4] == 1."""
    import torch
    lbm = lbm_lib
    L, raw = _state(lbm, precision)
    host = raw.cpu().numpy().copy()
    es = ESIZE[precision]
    n_cells = host.size // (27 * es)
    # population 5 of the first cell of the second 64-cell block: a stored fluid cell
    # in the compact layout or padding; either way one slot of one cell
    pos = (5 * n_cells + 64) * es
    nan = np.array([np.nan], dtype=np.float32 if es == 4 else np.float64)
    if precision == "bf16":
        host[pos:pos + 2] = np.frombuffer(np.array([0x7FC0], dtype="<u2").tobytes(), dtype=np.uint8)
    else:
        host[pos:pos + es] = np.frombuffer(nan.tobytes(), dtype=np.uint8)
    bad = torch.from_numpy(host).cuda()
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    lbm.lbm_reduce_static(bad, precision, 0, n_cells, out)
    torch.cuda.synchronize()
    assert out.cpu().numpy()[4] == 1
    L.close()


def test_static_reduce_rejects_bad_arguments(lbm_lib):
    import torch
    lbm = lbm_lib
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    buf = torch.zeros(27 * 4, dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_reduce_static(buf, "f32", 0, lbm.LBM_STATIC_REDUCE_MAX_CELLS + 1, out)
    assert ei.value.status == lbm.LBM_EINVAL
    assert "LBM_STATIC_REDUCE_MAX_CELLS" in str(ei.value)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_reduce_static(buf, "f32", 0, 0, out)
    with pytest.raises(lbm.LbmError) as ei:       # the output must be device memory
        lbm.lbm_reduce_static(buf, "f32", 0, 4, np.zeros(5))
    assert "out must be device" in str(ei.value)
    with pytest.raises(lbm.LbmError) as ei:       # so must the populations (refused before any launch)
        lbm.lbm_reduce_static(np.zeros(27 * 4, dtype=np.float32), "f32", 0, 4, out)
    assert ei.value.status == lbm.LBM_EINVAL and "pops must be device" in str(ei.value)
    torch.cuda.synchronize()
