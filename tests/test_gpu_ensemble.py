"""Batched ensemble, graph-captured chunks and launch shapes (GPU, through the C ABI).

* An ensemble member evolves bit-identically to the same pipe run alone (same kernel,
  same per-cell arithmetic; only the block-to-member map differs).
* Graph replays of captured step chunks equal direct launches bit for bit, statistics
  included.
* Every launch shape of the step kernel gives bit-identical populations.
* The autotuner leaves the state, the time and the statistics untouched.
* Two ensemble members in FP64 match the oracle run of each pipe to 1e-12.
"""
import math

import numpy as np
import pytest

from _pairs import make_pair, perturbed_state, rel_err
from paper_2405_12082_gb300 import workloads as Wk

pytestmark = pytest.mark.gpu

MEMBERS = [dict(R=5.0, nz=12, seed=11, phase=0.0, omega=1.7),
           dict(R=6.5, nz=16, seed=12, phase=1.1, omega=1.9),
           dict(R=8.3, nz=10, seed=13, phase=2.5, omega=1.5)]


def _member_setup(lbm, mem, precision="f32"):
    n = int(math.ceil(2 * mem["R"] + 4))
    grid = lbm.make_grid(n, n, mem["nz"], mem["R"], precision=precision, wall="halfway")
    trig = Wk.trigger_dict(h=3e-5, R=mem["R"], nz=mem["nz"], period=40.0,
                           modes=[(1, 0.5, mem["phase"]), (3, 0.5, 0.0)], t_end=15)
    force = lbm.make_force(g=(0.0, 0.0, 3e-5), trigger=trig)
    return grid, lbm.lbm_relax(mem["omega"]), force


def _populations(lbm, ctx, grid):
    f = np.empty((27, grid.nz, grid.ny, grid.nx))
    lbm.lbm_get_populations(ctx, f)
    return f


@pytest.mark.parametrize("graph", [0, 4])
def test_members_are_bit_identical_to_single_pipes(lbm_lib, graph):
    lbm = lbm_lib
    setups = [_member_setup(lbm, m) for m in MEMBERS]
    E = lbm.Lattice(None, None, ensemble=([s[0] for s in setups], [s[1] for s in setups], [s[2] for s in setups]))
    lbm.lbm_init(E.ctx, "laminar", noise_amp=1e-3, seed=500)
    if graph:
        lbm.lbm_set_graph(E.ctx, graph)
    E.step(21)
    for k, (grid, relax, force) in enumerate(setups):
        S = lbm.Lattice(grid, relax, force)
        lbm.lbm_init(S.ctx, "laminar", noise_amp=1e-3, seed=500 + k)    # member k draws seed + k
        S.step(21)
        E.select(k)
        a = _populations(lbm, E.ctx, grid)
        b = _populations(lbm, S.ctx, grid)
        assert np.array_equal(a, b), k
        S.close()
    E.close()


def test_graph_chunks_equal_direct_launches(lbm_lib):
    lbm = lbm_lib
    grid, relax, force = _member_setup(lbm, MEMBERS[1])
    runs = []
    for chunk in (0, 8):
        L = lbm.Lattice(grid, relax, force)
        lbm.lbm_init(L.ctx, "laminar", noise_amp=1e-3, seed=3)
        lbm.lbm_stats_enable(L.ctx, 4)
        if chunk:
            lbm.lbm_set_graph(L.ctx, chunk)
            assert L.info()["graph_chunk"] == chunk
        L.step(3)           # unaligned start: direct steps until t is a multiple of 4
        L.step(37)
        acc = np.empty((4, grid.nz, grid.ny, grid.nx))
        count = lbm.lbm_stats_get(L.ctx, acc)
        runs.append((_populations(lbm, L.ctx, grid), acc, count, L.info()["t"]))
        L.close()
    assert runs[0][3] == runs[1][3] == 40
    assert runs[0][2] == runs[1][2] == 10
    assert np.array_equal(runs[0][0], runs[1][0])
    assert np.array_equal(runs[0][1], runs[1][1])


def test_launch_shapes_agree(lbm_lib):
    lbm = lbm_lib
    grid, relax, force = _member_setup(lbm, MEMBERS[2])
    ref = None
    L = lbm.Lattice(grid, relax, force)
    nv = L.info()["n_variants"]
    L.close()
    # direct shapes, two software-pipelined persistent shapes, five with 2 or 4 planes per
    # thread, two staged persistent shapes
    assert nv == 13
    for v in range(nv):
        L = lbm.Lattice(grid, relax, force)
        lbm.lbm_set_variant(L.ctx, v)
        lbm.lbm_init(L.ctx, "laminar", noise_amp=1e-3, seed=9)
        L.step(9)
        f = _populations(lbm, L.ctx, grid)
        if ref is None:
            ref = f
        if v in (4, 5):
            # the pipelined kernel is compiled separately: the compiler may contract other
            # multiply-adds, so it agrees to FP32 rounding rather than bit for bit
            assert np.max(np.abs(f - ref)) <= 1e-6 * np.max(np.abs(ref)), v
        else:
            assert np.array_equal(f, ref), v
        L.close()
    L = lbm.Lattice(grid, relax, force)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_variant(L.ctx, nv)
    L.close()


def test_plane_coarsened_shapes_on_ragged_pipes(lbm_lib):
    """Shapes 6 and 7 (2 and 4 planes per thread) and the staged shapes 11 and 12 on an
    ensemble of two pipes whose length is not a multiple of 4: bit-identical to the
    one-cell-per-thread shape; in 16-bit storage the pipelined shapes are refused."""
    lbm = lbm_lib
    for prec in ("f32", "f16s"):
        grids = [lbm.make_grid(20, 20, 7, 8.3, precision=prec), lbm.make_grid(16, 18, 5, 6.1, precision=prec)]
        relaxes = [lbm.lbm_relax(1.3), lbm.lbm_relax(1.6)]
        forces = [lbm.make_force(g=(0, 0, 1e-5)), lbm.make_force(g=(1e-6, 0, 2e-5))]
        ref = None
        for v in (2, 6, 7, 8, 9, 10, 11, 12):
            E = lbm.Lattice(None, None, ensemble=(grids, relaxes, forces))
            lbm.lbm_set_variant(E.ctx, v)
            lbm.lbm_init(E.ctx, "laminar", noise_amp=1e-3, seed=21)
            E.step(7)
            out = []
            for k in range(2):
                E.select(k)
                out.append(E.populations())
            if ref is None:
                ref = out
            for k in range(2):
                assert np.array_equal(out[k], ref[k]), (prec, v, k)
            if prec == "f16s":
                for bad in (4, 5):
                    with pytest.raises(lbm.LbmError):
                        lbm.lbm_set_variant(E.ctx, bad)
            E.close()


def test_autotune_leaves_the_state_untouched(lbm_lib):
    lbm = lbm_lib
    grid, relax, force = _member_setup(lbm, MEMBERS[0])
    L = lbm.Lattice(grid, relax, force)
    lbm.lbm_init(L.ctx, "laminar", noise_amp=1e-3, seed=4)
    lbm.lbm_stats_enable(L.ctx, 2)
    L.step(5)
    before = _populations(lbm, L.ctx, grid)
    acc0 = np.empty((4, grid.nz, grid.ny, grid.nx))
    c0 = lbm.lbm_stats_get(L.ctx, acc0)
    v, us = lbm.lbm_autotune(L.ctx, 6)
    assert 0 <= v < 13 and us > 0
    info = L.info()
    assert info["t"] == 5 and info["variant"] == v and 0 <= info["variant_odd"] < 13
    assert np.array_equal(_populations(lbm, L.ctx, grid), before)
    acc1 = np.empty_like(acc0)
    assert lbm.lbm_stats_get(L.ctx, acc1) == c0
    assert np.array_equal(acc0, acc1)
    L.close()


def test_two_members_match_the_oracle_fp64(lbm_lib):
    lbm = lbm_lib
    pairs = []
    grids, relaxes, forces = [], [], []
    for k, mem in enumerate(MEMBERS[:2]):
        n = int(math.ceil(2 * mem["R"] + 4))
        L, ref = make_pair(lbm, n, n, mem["nz"], mem["R"], precision="f64", wall="halfway", omega=mem["omega"],
                           g=(0, 0, 3e-5), trigger=dict(h=3e-5, period=40.0,
                                                        modes=[(1, 0.5, mem["phase"]), (3, 0.5, 0.0)], t_end=15))
        f0 = perturbed_state(ref, 700 + k)
        pairs.append((ref, f0))
        grids.append(L.grid)
        relaxes.append(lbm.lbm_relax(mem["omega"]))
        forces.append(L._keep[0])
        L._keep.append((grids, forces))
        pairs[-1] = (ref, f0, L)
    E = lbm.Lattice(None, None, ensemble=(grids, relaxes, forces))
    for k, (ref, f0, _) in enumerate(pairs):
        E.select(k)
        E.set_populations(f0)
    E.step(12)
    for k, (ref, f0, L) in enumerate(pairs):
        ref.step(12)
        E.select(k)
        assert rel_err(E.populations(), ref.f, ref.fluid) < 1e-12
        L.close()
    E.close()


@pytest.mark.parametrize("graph", [0, 4])
def test_per_parity_shapes_are_bit_identical(lbm_lib, graph):
    """Different launch shapes for the even and the odd steps (lbm_set_variants), direct and
    in captured graphs (whose two parities then have different block counts), with
    statistics on: the same populations and sums as one shape for both."""
    lbm = lbm_lib
    grid, relax, force = _member_setup(lbm, MEMBERS[1])
    out = []
    for even, odd in ((6, 6), (6, 9), (2, 11), (12, 7), (9, 0)):
        L = lbm.Lattice(grid, relax, force)
        lbm.lbm_set_variants(L.ctx, even, odd)
        info = L.info()
        assert (info["variant"], info["variant_odd"]) == (even, odd)
        lbm.lbm_init(L.ctx, "laminar", noise_amp=1e-3, seed=9)
        lbm.lbm_stats_enable(L.ctx, 2)
        if graph:
            lbm.lbm_set_graph(L.ctx, graph)
        L.step(11)
        acc = np.empty((4, grid.nz, grid.ny, grid.nx))
        lbm.lbm_stats_get(L.ctx, acc)
        out.append((_populations(lbm, L.ctx, grid), acc))
        L.close()
    for f, acc in out[1:]:
        assert np.array_equal(f, out[0][0])
        assert np.array_equal(acc, out[0][1])
    L = lbm.Lattice(grid, relax, force)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_set_variants(L.ctx, 6, 99)
    assert (L.info()["variant"], L.info()["variant_odd"]) == (6, 9)      # unchanged defaults (F32)
    L.close()
