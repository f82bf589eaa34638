"""The C-ABI library loads and exports every function include/lbm.h declares; host-side
argument validation answers LBM_EINVAL before touching the GPU (no compute calls)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbm.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("lbm_create", "lbm_step", "lbm_moments", "lbm_free", "lbm_modes", "lbm_stats_enable",
                 "lbm_adjoint", "lbm_ensemble_create", "lbm_reduce"):
        assert must in names


def test_library_exports_every_declared_symbol(lbm_lib):
    lib = ctypes.CDLL(lbm_lib.LIB_PATH)
    for name in declared_functions():
        assert hasattr(lib, name), name
    assert set(declared_functions()) == set(lbm_lib.EXPORTED)


def _expect_einval(lbm, fn):
    with pytest.raises(lbm.LbmError) as ei:
        fn()
    assert ei.value.status == lbm.LBM_EINVAL
    return str(ei.value)


def test_create_rejects_bad_arguments_on_the_host(lbm_lib):
    lbm = lbm_lib
    relax = lbm.lbm_relax(1.2)
    msg = _expect_einval(lbm, lambda: lbm.lbm_create(lbm.make_grid(0, 10, 10, 3.0), relax))
    assert "sizes" in msg
    msg = _expect_einval(lbm, lambda: lbm.lbm_create(lbm.make_grid(10, 10, 10, 5.0), relax))
    assert "margin" in msg
    _expect_einval(lbm, lambda: lbm.lbm_create(lbm.make_grid(10, 10, 10, 3.0), lbm.lbm_relax(2.5)))
    _expect_einval(lbm, lambda: lbm.lbm_create(lbm.make_grid(10, 10, 10, 3.0, precision=7), relax))
    _expect_einval(lbm, lambda: lbm.lbm_create(lbm.make_grid(10, 10, 10, 3.0, wall=9), relax))
    _expect_einval(lbm, lambda: lbm.lbm_create(lbm.make_grid(10, 10, 10, -1.0), relax))
    bad = lbm.make_force(g=(0, 0, 1e-6), trigger=dict(A0=50, kappa=0.5, kz=3, l0=1, l=2, period=0, h=1e-6,
                                                    modes=[(2, 1, 0)]))
    msg = _expect_einval(lbm, lambda: lbm.lbm_create(lbm.make_grid(10, 10, 10, 3.0), relax, bad))
    assert "period" in msg
    assert "period" in lbm.lbm_last_error(None)


def test_struct_layouts_match_the_header(lbm_lib):
    """Sizes of the ctypes mirrors equal the C layouts (natural alignment, LP64)."""
    lbm = lbm_lib
    assert ctypes.sizeof(lbm.lbm_grid) == 40
    assert ctypes.sizeof(lbm.lbm_relax) == 16
    assert ctypes.sizeof(lbm.lbm_force) == 264
    assert ctypes.sizeof(lbm.lbm_modes_cfg) == 144
    assert ctypes.sizeof(lbm.lbm_info) == 72


def test_struct_layouts_match_a_c_compiler(lbm_lib, tmp_path):
    """Compile a probe against include/lbm.h and compare sizeof/offsetof with ctypes."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lbm = lbm_lib
    checks = {
        "lbm_grid": ["nx", "R", "precision", "wall", "f16_log2_scale"],
        "lbm_relax": ["omega", "rates"],
        "lbm_force": ["g", "trigger", "n_modes", "k_theta", "weight", "phase", "A0", "h", "kz", "t_end", "gz_field"],
        "lbm_modes_cfg": ["n_sections", "r_over_R", "n_theta", "n_modes"],
        "lbm_info": ["n_cells", "population_bytes", "n_members", "precision", "launches", "variant", "graph_chunk",
                     "variant_odd"],
    }
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "lbm.h"', "int main(void){"]
    for st, fields in checks.items():
        lines.append('printf("%s %%zu\\n", sizeof(%s));' % (st, st))
        for f in fields:
            lines.append('printf("%s.%s %%zu\\n", offsetof(%s, %s));' % (st, f, st, f))
    lines.append("return 0;}")
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = dict(line.split() for line in out if line.strip())
    for st, fields in checks.items():
        cls = getattr(lbm, st)
        assert int(got[st]) == ctypes.sizeof(cls), st
        for f in fields:
            assert int(got["%s.%s" % (st, f)]) == getattr(cls, f).offset, (st, f)


def test_create_reports_unsupported_sizes_on_the_host(lbm_lib):
    """27 x cells beyond 2^32 cannot be indexed by the step kernels: LBM_EUNSUPPORTED before
    any device allocation."""
    lbm = lbm_lib
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(lbm.make_grid(1000, 1000, 200, 0.0, geometry="box"), lbm.lbm_relax(1.2))
    assert ei.value.status == lbm.LBM_EUNSUPPORTED
    assert "32-bit" in str(ei.value)


def test_allocator_hooks_need_both_or_neither(lbm_lib):
    import ctypes as C
    lbm = lbm_lib
    a = lbm.ALLOC_FN(lambda n, s, u: 0)
    rc = lbm.LIB.lbm_set_allocator(a, C.cast(None, lbm.FREE_FN), None)
    assert rc == lbm.LBM_EINVAL
    assert "both" in lbm.lbm_last_error(None)
    lbm.lbm_set_allocator()           # both NULL: the default, accepted without a GPU


def test_fp32_probe_rejects_a_null_output_on_the_host(lbm_lib):
    lbm = lbm_lib
    assert lbm.LIB.lbm_probe_fp32(None, None) == lbm.LBM_EINVAL
    assert "out" in lbm.lbm_last_error(None)
