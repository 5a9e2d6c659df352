"""The C ABI library loads and exports every symbol include/gmead.h declares;
host-side argument checks work without a GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_1708_09705_gb300 import _build
    _build.build()
    import paper_1708_09705_gb300 as gm
    return gm.lib()


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "gmead.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(gm_[a-z_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(L):
    names = declared_symbols()
    assert len(names) >= 15
    for name in names:
        assert hasattr(L, name), name
    import paper_1708_09705_gb300 as gm
    assert sorted(gm.EXPORTS) == names


def test_status_strings_and_defaults(L):
    import paper_1708_09705_gb300 as gm
    assert L.gm_status_str(0) == b"GM_OK"
    assert L.gm_status_str(4) == b"GM_E_NOT_SPD"
    cfg = gm.default_config()
    assert cfg.sigma2 == 1.0 and cfg.outer_scale_pc == 20.0 and cfg.cutoff_pc == 60.0
    assert cfg.precision == gm.PREC_FP64 and cfg.taper == gm.TAPER_WENDLAND
    assert cfg.warm_start == 1 and cfg.rhs_panel == 0
    assert C.sizeof(gm.Config) == 8 * 4 + 4 * 6 + 8 * 3 + 4 * 2 + 4 * 2 + 8 + 8 + 8
    assert cfg.cov_source == gm.COV_QUADRATURE and cfg.surrogate_gate == 1e-4
    assert cfg.probe_factor == 0.0        # exact variances unless asked
    assert cfg.deflate == 0
    assert cfg.quad_rule == gm.QUAD_BAND and cfg.tc_products == 6   # the converged rule


def test_init_rejects_bad_arguments_before_touching_a_gpu(L):
    import paper_1708_09705_gb300 as gm
    h = C.c_void_p()
    x = (C.c_double * 4)(1, 2, 3, 4)
    cfg = gm.default_config()
    # n = 0
    assert L.gm_ep_init(C.byref(h), C.byref(cfg), 0, x, x, x, x, x, None, None) == 1
    # null array
    assert L.gm_ep_init(C.byref(h), C.byref(cfg), 4, x, None, x, x, x, None, None) == 1
    for field, bad in (("sigma2", -1.0), ("n_nodes", 1), ("damping", 0.0), ("cg_tol", 0.0),
                       ("precision", 7), ("outer_scale_pc", float("nan")), ("warm_start", 2),
                       ("probe_factor", -1.0), ("probe_factor", float("inf")),
                       ("deflate", 5), ("deflate", -64), ("quad_rule", 2),
                       ("tc_products", 4)):
        c2 = gm.default_config(**{field: bad})
        assert L.gm_ep_init(C.byref(h), C.byref(c2), 4, x, x, x, x, x, None, None) == 1, field
    assert not h.value
    # several fields: field ids required, FP32 form only, positive field scales
    fid = (C.c_int32 * 4)(0, 1, 0, 1)
    L0 = (C.c_double * 2)(20.0, -1.0)
    c32 = gm.default_config(precision=gm.PREC_FP32)
    assert L.gm_ep_init_fields(C.byref(h), C.byref(c32), 4, x, x, x, x, x, 2, None, None, None,
                               None, None) == 1
    assert L.gm_ep_init_fields(C.byref(h), C.byref(cfg), 4, x, x, x, x, x, 2, fid, None, None,
                               None, None) == 1
    assert L.gm_ep_init_fields(C.byref(h), C.byref(c32), 4, x, x, x, x, x, 2, fid, L0, None,
                               None, None) == 1
    assert not h.value
    # calls on a null context
    assert L.gm_build_cov(None, None) == 1
    assert L.gm_ep_sweep(None, 1, 0.0, None, None) == 1
    assert L.gm_predict_sightlines(None, 1, 2, x, x, x, x, x) == 1
    assert L.gm_monotone_sample(None, 1, 2, x, x, x, 0, 1, x, None) == 1
    blk = (C.c_int32 * 4)(0, 0, 1, 1)
    assert L.gm_pic_posterior(None, 2, blk, 2, x, x, x, x, x) == 1
    assert L.gm_pic_predict(None, 2, blk, x, x, x, x, x) == 1


def test_header_is_plain_c99(tmp_path):
    """include/gmead.h is a C header: it compiles as strict C99 (no C++ in the
    declarations, fixed-width types only)."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "gmead.h"\n'
                   "int main(void) { gm_config c; gm_stats s;\n"
                   "  gm_config_default(&c); s.nnz = 0;\n"
                   "  return c.n_nodes < 0 || s.nnz != 0; }\n")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    f"-I{os.path.join(ROOT, 'include')}", "-c", str(src), "-o",
                    str(tmp_path / "use.o")], check=True)
