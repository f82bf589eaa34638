"""Device-memory hooks (lbm_set_allocator): every device buffer of a context comes from the
caller's allocator and goes back to it, results do not depend on where the memory came
from, and a failing or misaligned hook is reported as LBM_ENOMEM."""
import numpy as np
import pytest

from _pairs import make_pair, perturbed_state, rel_err
from paper_2405_12082_gb300 import workloads as Wk

pytestmark = pytest.mark.gpu


class Recorder:
    """Hooks backed by PyTorch's caching allocator that remember what is live."""

    def __init__(self, offset=0):
        self.live = {}
        self.n_alloc = 0
        self.offset = offset

    def alloc(self, nbytes, stream):
        import torch
        base = torch.cuda.caching_allocator_alloc(nbytes + self.offset, torch.cuda.current_device(), stream)
        self.n_alloc += 1
        self.live[base + self.offset] = base
        return base + self.offset

    def free(self, ptr, stream):
        import torch
        torch.cuda.caching_allocator_delete(self.live.pop(ptr))


def _run(lbm, use_hooks, rec=None):
    if use_hooks:
        lbm.lbm_set_allocator(rec.alloc, rec.free)
    try:
        L, ref = make_pair(lbm, 20, 20, 8, 8.2, precision="f64", omega=1.4, g=(0, 0, 2e-5))
        gz = Wk.gz_field(8, 20, 20, base=2e-5, seed=31, rel_amp=0.2)
        f0 = perturbed_state(ref, 611)
        L.set_populations(f0)                       # host input: staging buffer
        lbm.lbm_stats_enable(L.ctx, 2)              # statistics accumulators
        lbm.lbm_set_graph(L.ctx, 4)                 # graph step tables
        L.step(8)
        lbm.lbm_set_graph(L.ctx, 0)
        acc = np.empty((4, 8, 20, 20))
        lbm.lbm_stats_get(L.ctx, acc)
        J, dw = lbm.lbm_adjoint(L.ctx, 6, lbm.LBM_J_UBULK, 2, np.zeros((8, 20, 20)))   # adjoint temporaries
        f = L.populations()
        L.close()
        return f, acc, J, dw
    finally:
        if use_hooks:
            lbm.lbm_set_allocator()


def test_hooks_own_every_buffer_and_change_nothing(lbm_lib):
    lbm = lbm_lib
    rec = Recorder()
    a = _run(lbm, False)
    b = _run(lbm, True, rec)
    assert rec.n_alloc >= 6                 # populations, members, partials, tables, stats, staging, ...
    assert rec.live == {}                   # everything went back
    assert np.array_equal(a[0], b[0])
    assert np.array_equal(a[1], b[1])
    assert a[2] == b[2] and a[3] == b[3]


def test_torch_caching_allocator_backs_a_context(lbm_lib):
    import torch
    lbm = lbm_lib
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    lbm.use_torch_allocator()
    try:
        L, ref = make_pair(lbm, 24, 24, 16, 10.0, precision="f32", omega=1.3)
        during = torch.cuda.memory_allocated()
        assert during - before >= L.info()["population_bytes"]
        L.init("laminar", noise_amp=1e-3, seed=2)
        ref.init("laminar", noise_amp=1e-3, seed=2)
        L.step(5)
        ref.step(5)
        assert rel_err(L.populations(), ref.f, ref.fluid) < 1e-6
        L.close()
    finally:
        lbm.lbm_set_allocator()
    torch.cuda.synchronize()
    assert torch.cuda.memory_allocated() == before


def test_failing_and_misaligned_hooks_are_out_of_memory(lbm_lib):
    lbm = lbm_lib
    grid = lbm.make_grid(12, 12, 4, 4.5, precision="f32")
    lbm.lbm_set_allocator(lambda n, s: 0, lambda p, s: None)
    try:
        with pytest.raises(lbm.LbmError) as e:
            lbm.Lattice(grid, lbm.lbm_relax(1.2))
        assert e.value.status == lbm.LBM_ENOMEM
    finally:
        lbm.lbm_set_allocator()
    rec = Recorder(offset=16)
    lbm.lbm_set_allocator(rec.alloc, rec.free)
    try:
        with pytest.raises(lbm.LbmError) as e:
            lbm.Lattice(grid, lbm.lbm_relax(1.2))
        assert e.value.status == lbm.LBM_ENOMEM
    finally:
        lbm.lbm_set_allocator()
    assert rec.live == {}                   # the misaligned block was handed back
