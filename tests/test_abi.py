"""The C-ABI library builds, loads and exports every declared symbol (no GPU)."""

import ctypes
import glob
import os
import re

import numpy as np
import pytest

import paper_2310_13908_gb300 as sk
from paper_2310_13908_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                             text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "for", "while", "return", "sizeof", "defined"):
                names.add(name)
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return sk.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("sk_create", "sk_destroy", "sk_last_error", "stokes_sl_eval",
                     "stokes_dl_eval"):
        assert required in names


def test_every_entry_point_cites_its_passage():
    """Each declaration's own comment, or the header comment of its section,
    cites the paper (Sec., Eq., Table, Appendix) or states that the paper has
    no counterpart (library infrastructure)."""
    cite = re.compile(r"Sec\.|Eq\.|Table|Appendix|defines no API|no counterpart")
    decl = re.compile(r"^(?:int|void|const char\*)\s+\**(\w+)\s*\(", re.M)
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        body = text[text.index("#ifndef"):]
        sections = [m.start() for m in re.finditer(r"/\* ---- ", body)]
        prev_end, seen = 0, set()
        for m in decl.finditer(body):
            own = body[prev_end:m.start()]
            starts = [p for p in sections if p <= m.start()]
            head = body[starts[-1]:body.index("*/", starts[-1]) + 2] if starts else ""
            assert cite.search(own) or cite.search(head), f"{os.path.basename(h)}: {m.group(1)}"
            prev_end = body.index(";", m.start()) + 1
            seen.add(m.group(1))
        # every declared function was checked
        assert seen == set(declared_functions())


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_version_and_null_context_rejections(lib):
    assert sk.sk_version() == 100
    # argument checks that return before any CUDA call
    assert lib.stokes_sl_eval(None, 1, 0, 0, None, None, None, 1, None, None, 1, 1.0, None,
                              None) == sk.SK_EINVAL
    assert lib.sk_create(None, 0, 0) == sk.SK_EINVAL
    assert lib.sk_set_fp32c_thresholds(None, 0.5, 5.0) == sk.SK_EINVAL


def test_library_fails_loudly_when_missing(monkeypatch, tmp_path):
    monkeypatch.setattr(sk, "_lib", None)
    monkeypatch.setattr(sk, "LIB_PATH", str(tmp_path / "libstokesreg.so"))
    with pytest.raises(RuntimeError, match="build the CUDA library"):
        sk.load()


def test_build_flags_target_sm103a():
    assert "arch=compute_103a,code=sm_103a" in _build.ARCH


def test_serving_entry_points_reject_null_arguments(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.serve_create(None, None, ctypes.byref(h)) == sk.SK_EINVAL
    t = ctypes.c_uint64()
    assert lib.serve_submit(None, None, ctypes.byref(t)) == sk.SK_EINVAL
    assert lib.serve_poll(None, ctypes.c_uint64(1), None, None, 0) == sk.SK_EINVAL
    lib.serve_destroy(None)  # no-op


def test_capsule_entry_points_reject_null_arguments(lib):
    import ctypes
    h = ctypes.c_void_p()
    assert lib.capsule_create(None, ctypes.byref(h), 9, None, None, None, 0, 1.0, 1) == sk.SK_EINVAL
    assert lib.capsule_step(None, 1, 0.1, None, None) == sk.SK_EINVAL
    assert lib.capsule_get(None, None) == sk.SK_EINVAL
    assert lib.capsule_set_membrane(None, None, 1.0, 1.0) == sk.SK_EINVAL
    assert lib.capsule_area_volume(None, None, None) == sk.SK_EINVAL
    assert lib.capsule_integrate_rkf45(None, 1.0, None, 1e-6, None, None, 10, None) == sk.SK_EINVAL
    lib.capsule_destroy(None)  # no-op


def test_membrane_entry_points_reject_null_context(lib):
    assert lib.surface_derivatives(None, 9, sk.SK_HOST, 1, None, None, None, None) == sk.SK_EINVAL
    assert lib.membrane_force(None, 9, sk.SK_HOST, None, None, 1.0, 1.0, None, None,
                              None) == sk.SK_EINVAL
    assert lib.stokes_sl_eval_upsampled(None, sk.SK_FP64, sk.SK_HOST, 9, None, None, None, 1.0,
                                        None, None) == sk.SK_EINVAL
    assert lib.stokes_sl_eval_fmm(None, sk.SK_FP64, sk.SK_HOST, 1, None, None, None, 1, None, None,
                                  1, 1.0, 1, None, 1, 4, None, None) == sk.SK_EINVAL


def test_probe_and_stats_entry_points_reject_null_arguments(lib):
    assert lib.sk_probe_peaks(None, None) == sk.SK_EINVAL
    assert lib.sk_last_eval_stats(None, None) == sk.SK_EINVAL
    assert lib.sk_set_profiling(None, 1) == sk.SK_EINVAL
    assert lib.capsule_set_upsampling(None, 4) == sk.SK_EINVAL
    assert lib.capsule_shape_moments(None, None) == sk.SK_EINVAL


def test_host_arrays_with_the_wrong_shape_are_rejected(lib):
    # checked in the binding, before any CUDA call
    X = np.zeros((12, 4))          # 48 values: would reshape to (16, 3) silently
    with pytest.raises(ValueError, match="src_xyz"):
        sk.stokes_sl_eval(None, sk.SK_FP32C, sk.SK_HOST, X, np.ones(12), np.ones((12, 3)),
                          np.zeros((2, 3)), 0.1)
    with pytest.raises(ValueError, match="src_w"):
        sk.stokes_sl_eval(None, sk.SK_FP32C, sk.SK_HOST, np.zeros((12, 3)), np.ones((12, 2)),
                          np.ones((12, 3)), np.zeros((2, 3)), 0.1)


def test_header_is_plain_c(tmp_path):
    """include/stokesreg.h is a C ABI: it compiles as C99 (no C++ in it)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "use.c"
    src.write_text('#include "stokesreg.h"\nint main(void) { return sk_version() > 0 ? 0 : 1; }\n')
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-fsyntax-only",
                        "-I", inc, str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


def test_c_program_links_and_runs(lib, tmp_path):
    """A plain C program built against the header links with libstokesreg.so
    alone and runs: sk_create returns SK_OK on a GPU, SK_ECUDA (with a message)
    where there is no CUDA driver."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(sk.LIB_PATH)
    src = tmp_path / "use.c"
    src.write_text(
        '#include <stdio.h>\n#include "stokesreg.h"\n'
        "int main(void) {\n"
        "  sk_ctx* ctx = NULL;\n"
        "  int rc = sk_create(&ctx, 0, 0);\n"
        '  printf("%d %s\\n", rc, rc == SK_OK ? "" : sk_last_error(NULL));\n'
        "  if (rc == SK_OK) sk_destroy(ctx);\n"
        "  return 0;\n}\n")
    exe = tmp_path / "use"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                        str(src), "-L", libdir, "-lstokesreg", f"-Wl,-rpath,{libdir}", "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr
    code = int(r.stdout.split()[0])
    assert code in (sk.SK_OK, sk.SK_ECUDA), r.stdout


@pytest.mark.gpu
def test_c_program_evaluates_the_self_limit(lib, tmp_path):
    """A plain C program evaluates stokes_sl_eval through the ABI alone, in
    both precisions, on host arrays: one source with a target on it gives the
    r -> 0 limit of Sec. 3.4, u = w f / (8 pi mu) * 16 / (3 delta sqrt(pi)),
    and a distant target the textbook Stokeslet of Sec. 2.2 to O(e^-rho^2)."""
    import shutil
    import subprocess
    gcc = shutil.which("gcc") or shutil.which("cc")
    if gcc is None:
        pytest.skip("no C compiler")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    libdir = os.path.dirname(sk.LIB_PATH)
    src = tmp_path / "eval.c"
    src.write_text(r"""
#include <math.h>
#include <stdio.h>
#include "stokesreg.h"
int main(void) {
  sk_ctx* ctx = NULL;
  if (sk_create(&ctx, 0, 0) != SK_OK) { printf("create %s\n", sk_last_error(NULL)); return 2; }
  const double x[3] = {1.0, 2.0, 3.0}, w[1] = {0.7}, f[3] = {0.3, -1.2, 2.0};
  const double y[6] = {1.0, 2.0, 3.0, 1.0, 2.0, 13.0};  /* on the node; 10 away on z */
  const double delta = 0.2, mu = 1.5, pi = 3.14159265358979323846;
  const int precs[2] = {SK_FP64, SK_FP32C};
  int bad = 0;
  for (int k = 0; k < 2; ++k) {
    double u[6];
    int rc = stokes_sl_eval(ctx, precs[k], SK_HOST, 1, x, w, f, 2, y, &delta, 1, mu, u, NULL);
    if (rc != SK_OK) { printf("eval %d %s\n", rc, sk_last_error(ctx)); return 3; }
    const double lim = 16.0 / (3.0 * delta * sqrt(pi)) * w[0] / (8.0 * pi * mu);
    const double tol = k == 0 ? 1e-13 : 1e-12;
    for (int c = 0; c < 3; ++c) {
      const double ref = lim * f[c];
      if (fabs(u[c] - ref) > tol * fabs(ref)) { printf("self %d %d %.17g %.17g\n", k, c, u[c], ref); bad = 1; }
    }
    /* d = (0, 0, 10): u = w / (8 pi mu) (f / r + (f . d) d / r^3) */
    const double r = 10.0, s = w[0] / (8.0 * pi * mu);
    const double far[3] = {s * f[0] / r, s * f[1] / r, s * (f[2] / r + f[2] * 100.0 / (r * r * r))};
    const double tf = k == 0 ? 1e-13 : 1e-6;
    for (int c = 0; c < 3; ++c)
      if (fabs(u[3 + c] - far[c]) > tf * fabs(far[2])) { printf("far %d %d %.17g %.17g\n", k, c, u[3 + c], far[c]); bad = 1; }
  }
  sk_destroy(ctx);
  printf("%s\n", bad ? "FAIL" : "OK");
  return bad;
}
""")
    exe = tmp_path / "eval"
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(root, "include"),
                        str(src), "-L", libdir, "-lstokesreg", f"-Wl,-rpath,{libdir}", "-lm",
                        "-o", str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("OK")
