"""The staged step kernel (launch shapes 11 and 12: populations of whole row groups copied
into shared memory with bulk copies several tiles ahead) through the C ABI.

* FP64 storage: against the FP64 oracle after 1-3 steps from non-equilibrium states, for
  half-way and Bouzidi walls and both AA parities, on a ragged box (1e-13, as the direct
  shapes).
* Bit-identical to the default direct shape: with statistics on, in graph-captured chunks,
  in every storage on the full-size R = 96 pipe and on the 16-pipe ensemble.
* Refused where it cannot run: full-way walls and the periodic box (no compact rows), and
  a pipe whose widest row does not fit the shape's shared-memory segments.
* Failure detection: a tile whose copies are never issued makes its CTA's bounded wait
  expire; the context reports LBM_ETIMEOUT and stays usable.
"""
import math

import numpy as np
import pytest

from _pairs import TRIG_MODES, make_pair, perturbed_state, rel_err
from paper_2405_12082_gb300 import workloads as Wk

pytestmark = pytest.mark.gpu

STAGED = (11, 12)


@pytest.mark.parametrize("variant", STAGED)
@pytest.mark.parametrize("wall", ["halfway", "bouzidi"])
@pytest.mark.parametrize("steps", [1, 2, 3])
def test_fp64_staged_step_matches_the_oracle(lbm_lib, variant, wall, steps):
    L, ref = make_pair(lbm_lib, 23, 19, 7, 7.3, precision="f64", wall=wall, omega=1.7, g=(2e-5, -1e-5, 3e-5),
                       trigger=dict(h=1e-4, period=30.0, modes=TRIG_MODES, t_end=9))
    lbm_lib.lbm_set_variant(L.ctx, variant)
    f0 = perturbed_state(ref, 111)
    L.set_populations(f0)
    L.step(steps)
    ref.step(steps)
    assert rel_err(L.populations(), ref.f, ref.fluid) < 1e-13
    L.close()


def _pipe(lbm, nx, nz, R, precision="f32", wall="halfway", stats=0):
    grid = lbm.make_grid(nx, nx, nz, R, precision=precision, wall=wall)
    trig = Wk.trigger_dict(h=2e-5, R=R, nz=nz, period=25.0, modes=TRIG_MODES, t_end=40)
    L = lbm.Lattice(grid, lbm.lbm_relax(1.8), lbm.make_force(g=(0.0, 0.0, 2e-5), trigger=trig))
    L.init("laminar", noise_amp=2e-3, seed=31)
    if stats:
        lbm.lbm_stats_enable(L.ctx, stats)
    return L


def _raw(lbm, L):
    import torch
    n = L.info()["population_bytes"]
    buf = torch.empty(n, dtype=torch.uint8, device="cuda")
    lbm.lbm_get_raw(L.ctx, buf, n)
    return buf


@pytest.mark.parametrize("precision", ["f32", "f16s", "bf16", "f64"])
@pytest.mark.parametrize("wall", ["halfway", "bouzidi"])
def test_staged_shapes_are_bit_identical_with_statistics_and_graphs(lbm_lib, precision, wall):
    import torch
    lbm = lbm_lib
    out = {}
    for v in (None,) + STAGED:
        for graph in (0, 6):
            L = _pipe(lbm, 30, 11, 12.7, precision, wall, stats=3)
            if v is not None:
                lbm.lbm_set_variant(L.ctx, v)
            if graph:
                lbm.lbm_set_graph(L.ctx, graph)
            L.step(13)
            acc = torch.empty((4, 11, 30, 30), dtype=torch.float64, device="cuda")
            count = lbm.lbm_stats_get(L.ctx, acc)
            out[(v, graph)] = (_raw(lbm, L), acc, count)
            assert lbm.lbm_reduce(L.ctx)[4] == 0
            L.close()
    r0, a0, c0 = out[(None, 0)]
    for key, (r, a, c) in out.items():
        assert torch.equal(r, r0), key
        assert torch.equal(a, a0) and c == c0, key


@pytest.mark.parametrize("precision", ["f32", "f16s", "bf16"])
def test_staged_shape_bit_identical_on_the_large_pipe(lbm_lib, precision):
    """The R = 96, 196 x 196 x 1152 pipe (69 k tiles, every SM looping over its share) with
    the four-mode trigger: 4 steps from the same start in the default shape and in each
    staged shape give the same bytes."""
    import torch
    lbm = lbm_lib
    cfg = Wk.C3
    raws = []
    for v in (None,) + STAGED:
        grid = lbm.make_grid(cfg["nx"], cfg["ny"], cfg["nz"], cfg["R"], precision=precision, wall="halfway")
        trig = Wk.trigger_dict(h=cfg["h"], R=cfg["R"], nz=cfg["nz"], period=cfg["period"],
                               modes=cfg["trigger_modes"], t_end=cfg["t_trigger"])
        L = lbm.Lattice(grid, lbm.lbm_relax(cfg["omega"]), lbm.make_force(g=(0.0, 0.0, cfg["h"]), trigger=trig))
        if v is not None:
            lbm.lbm_set_variant(L.ctx, v)
        L.init("loglaw", noise_amp=cfg["noise"], seed=Wk.SEED)
        L.step(4)
        raws.append(_raw(lbm, L))
        assert lbm.lbm_reduce(L.ctx)[4] == 0
        L.close()
    for k in range(1, len(raws)):
        assert torch.equal(raws[k], raws[0]), (precision, k)
    del raws
    torch.cuda.empty_cache()


def test_staged_shape_on_the_ensemble(lbm_lib):
    """The 16-pipe ensemble (4 radii, one flat tile list over all members): bit-identical to
    the default shape after 6 steps."""
    import torch
    lbm = lbm_lib
    cfg = Wk.C4
    members = Wk.ensemble_members(Wk.SEED, cfg["n"], cfg["radii"], cfg["u_star"])
    grids, relaxes, forces = [], [], []
    for mem in members:
        n = Wk.box_side(mem["R"])
        grids.append(lbm.make_grid(n, n, cfg["nz"], mem["R"], precision="f32", wall="halfway"))
        relaxes.append(lbm.lbm_relax(cfg["omega"]))
        forces.append(lbm.make_force(g=(0.0, 0.0, mem["h"]),
                                     trigger=Wk.trigger_dict(h=mem["h"], R=mem["R"], nz=cfg["nz"],
                                                             period=mem["period"], modes=[(2, 1.0, mem["phase"])],
                                                             t_end=mem["t_end"])))
    raws = []
    for v in (None, 11):
        E = lbm.Lattice(None, None, ensemble=(grids, relaxes, forces))
        if v is not None:
            lbm.lbm_set_variant(E.ctx, v)
        lbm.lbm_init(E.ctx, "loglaw", noise_amp=cfg["noise"], seed=Wk.SEED)
        E.step(6)
        raws.append(_raw(lbm, E))
        E.close()
    assert torch.equal(raws[0], raws[1])


def test_staged_shapes_are_refused_where_they_cannot_run(lbm_lib):
    lbm = lbm_lib
    for kw in (dict(wall="fullway"),):
        L = _pipe(lbm, 20, 6, 8.0, "f32", kw["wall"])
        for v in STAGED:
            with pytest.raises(lbm.LbmError) as ei:
                lbm.lbm_set_variant(L.ctx, v)
            assert ei.value.status == lbm.LBM_EUNSUPPORTED
        L.close()
    B = lbm.Lattice(lbm.make_grid(8, 8, 4, 0.0, geometry="box", precision="f32"), lbm.lbm_relax(1.2))
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_variant(B.ctx, 11)
    B.close()
    # rows of about 580 cells: wider than the 576-element segments of both staged shapes
    # in F32 storage, narrower than the 1088 of the 16-bit formats
    for prec, ok in (("f32", False), ("bf16", True)):
        L = _pipe(lbm, 584, 2, 290.0, prec)
        L.init("rest")                      # (a laminar start would be far beyond Mach 1 at this radius)
        for v in STAGED:
            if ok:
                lbm.lbm_set_variant(L.ctx, v)
                L.step(2)
                assert lbm.lbm_reduce(L.ctx)[4] == 0
            else:
                with pytest.raises(lbm.LbmError) as ei:
                    lbm.lbm_set_variant(L.ctx, v)
                assert ei.value.status == lbm.LBM_EUNSUPPORTED
        L.close()


def test_an_expired_wait_is_reported_and_the_context_stays_usable(lbm_lib):
    lbm = lbm_lib
    L = _pipe(lbm, 40, 16, 17.0, "f32")
    lbm.lbm_set_variant(L.ctx, 11)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_test_expire_wait(L.ctx, -1)
    assert ei.value.status == lbm.LBM_EINVAL
    lbm.lbm_test_expire_wait(L.ctx, 3)
    L.step(1)                                     # one CTA gives up on its fourth tile
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_reduce(L.ctx)
    assert ei.value.status == lbm.LBM_ETIMEOUT
    assert "bounded wait" in str(ei.value)
    # reported once; a fresh start then runs normally
    L.init("laminar", noise_amp=2e-3, seed=31)
    L.step(6)
    assert lbm.lbm_reduce(L.ctx)[4] == 0
    # the same through the periodic check
    lbm.lbm_set_check(L.ctx, 1, 1.0)
    lbm.lbm_test_expire_wait(L.ctx, 0)
    with pytest.raises(lbm.LbmError) as ei:
        L.step(1)
    assert ei.value.status == lbm.LBM_ETIMEOUT
    L.close()
    D = _pipe(lbm, 40, 16, 17.0, "f32")          # a direct shape has no staged tiles
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_test_expire_wait(D.ctx, 0)
    assert ei.value.status == lbm.LBM_EUNSUPPORTED
    D.close()
