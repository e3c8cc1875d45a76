"""Host-side checks of the C ABI: the library builds and loads, exports every
function include/gbmg.h declares, and the ctypes structures of the binding
match the C layout (sizes and field offsets measured by a gcc probe)."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gbmg.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(mg_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__
    __graft_entry__.build()
    import paper_1612_07873_gb300 as gb
    return C.CDLL(gb.LIB_PATH)


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_function():
    import paper_1612_07873_gb300 as gb
    names = declared_functions()
    missing = [n for n in names if n not in ("mg_default_params", "mg_status_string",
                                             "mg_last_error") and not hasattr(gb, n)]
    assert not missing, missing


def test_struct_layout_matches_c(tmp_path):
    import paper_1612_07873_gb300 as gb
    fields_p = [f for f, _ in gb.mg_params._fields_]
    fields_s = [f for f, _ in gb.mg_solve_stats._fields_]
    body = ['#include <stdio.h>', '#include <stddef.h>', '#include "gbmg.h"', "int main(void){",
            'printf("%zu %zu\\n", sizeof(mg_params), sizeof(mg_solve_stats));']
    body += [f'printf("%zu\\n", offsetof(mg_params, {f}));' for f in fields_p]
    body += [f'printf("%zu\\n", offsetof(mg_solve_stats, {f}));' for f in fields_s]
    body += ["return 0;}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(body))
    exe = tmp_path / "probe"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in out]
    assert vals[0] == C.sizeof(gb.mg_params)
    assert vals[1] == C.sizeof(gb.mg_solve_stats)
    offs = vals[2:]
    want = [getattr(gb.mg_params, f).offset for f in fields_p] + \
           [getattr(gb.mg_solve_stats, f).offset for f in fields_s]
    assert offs == want


def test_default_params_and_status_strings(lib):
    import paper_1612_07873_gb300 as gb
    p = gb.default_params(dims=(4, 4, 4, 4), block=[(2, 2, 2, 2)], nvec=[4], mass=-0.1)
    assert p.gcr_nkrylov == 10 and p.mr_iters == 4 and p.coarse_maxiter == 100
    assert tuple(p.dims) == (4, 4, 4, 4) and p.nvec[0] == 4
    for code in range(-8, 1):
        assert gb.LIB.mg_status_string(code)


def test_create_rejects_bad_arguments_without_a_gpu(lib):
    """Argument errors are reported before any device call."""
    import paper_1612_07873_gb300 as gb
    p = gb.default_params(dims=(4, 4, 4, 4), block=[(2, 2, 2, 2)], nvec=[4])
    h = C.c_void_p()
    assert gb.LIB.mg_create(C.byref(p), None, C.byref(h)) == gb.MG_ERR_ARG
    p.nlevels = 9
    assert gb.LIB.mg_create(C.byref(p), C.c_void_p(16), C.byref(h)) == gb.MG_ERR_ARG
    assert b"nlevels" in gb.LIB.mg_last_error(None)


def test_noalloc_rejects_bad_arguments_without_a_gpu(lib):
    """The allocation-free block orthonormalisation checks its arguments
    before any device call: the pointers below are never dereferenced."""
    import paper_1612_07873_gb300 as gb
    f = gb.LIB.mg_block_orthonormalise_noalloc
    a, b = C.c_void_p(256), C.c_void_p(512)

    def call(dims, block, ndof, nvec, x=a, y=b, nbytes=None):
        if nbytes is None:
            vol = 1
            for v in dims:
                vol *= v
            nbytes = nvec * vol * ndof * 16
        return f(x, y, nbytes, (C.c_int * 4)(*dims), (C.c_int * 4)(*block), ndof, nvec, None)

    big = 1 << 16   # 2^64 sites: the running volume product must not wrap
    cases = [
        (((4, 4, 4, 4), (2, 2, 2, 2), 12, 4, None, b), b"null"),
        (((4, 4, 4, 4), (2, 2, 2, 2), 12, 4, a, a), b"aliases"),
        (((4, 4, 4, 4), (2, 2, 2, 2), 11, 4), b"ndof"),
        (((4, 4, 4, 4), (2, 2, 2, 2), 12, 65), b"exceeds 64"),
        (((4, 4, 4, 6), (2, 2, 2, 4), 12, 4), b"divisible"),
        (((8, 8, 8, 8), (2, 2, 2, 2), 24, 24), b"2^21"),
        (((big, big, big, big), (1, 1, 1, 1), 12, 1, a, b, 16), b"2^21"),
        (((4, 4, 4, 4), (2, 2, 2, 2), 12, 4, a, b, 4 * 256 * 12 * 16 - 16), b"bytes"),
        (((4, 4, 4, 4), (2, 2, 2, 2), 12, 4, a, b, 0), b"bytes"),
    ]
    for args, text in cases:
        assert call(*args) == gb.MG_ERR_ARG, args
        assert text in gb.LIB.mg_last_error(None), (args, gb.LIB.mg_last_error(None))


def test_fma_peak_rejects_bad_arguments_without_a_gpu(lib):
    import paper_1612_07873_gb300 as gb
    t = C.c_double()
    assert gb.LIB.mg_fma_peak(gb.BF16, C.byref(t), None) == gb.MG_ERR_ARG
    assert b"prec" in gb.LIB.mg_last_error(None)
    assert gb.LIB.mg_fma_peak(gb.F32, None, None) == gb.MG_ERR_ARG


def test_tuner_cache_file_and_pins_without_a_gpu(lib, tmp_path):
    """The launch-policy cache (GBMG_TUNE_CACHE, "key value" lines) is read
    on first use; mg_tune_set pins or (choice < 0) clears a key.  Run in a
    fresh process, where the tuner reads its environment."""
    import sys
    cache = tmp_path / "tune.txt"
    cache.write_text("wilson/v4096/n1/c1 4\ncoarse/v256/n48 2\n")
    code = (
        "import ctypes as C, sys\n"
        "sys.path.insert(0, %r)\n"
        "import paper_1612_07873_gb300 as gb\n"
        "L = gb.LIB\n"
        "g = lambda k: L.mg_tune_get(k.encode())\n"
        "assert g('wilson/v4096/n1/c1') == 4 and g('coarse/v256/n48') == 2\n"
        "assert g('absent') == -1\n"
        "assert L.mg_tune_set(b'wilson/v4096/n1/c1', 7) == 0 and g('wilson/v4096/n1/c1') == 7\n"
        "assert L.mg_tune_set(b'coarse/v256/n48', -1) == 0 and g('coarse/v256/n48') == -1\n"
        "assert L.mg_tune_set(None, 1) == gb.MG_ERR_ARG and L.mg_tune_get(None) == -1\n"
        "print('ok')\n" % ROOT)
    env = dict(os.environ, GBMG_TUNE_CACHE=str(cache))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stderr
    # pins are not written back to the cache file
    assert cache.read_text() == "wilson/v4096/n1/c1 4\ncoarse/v256/n48 2\n"


@pytest.mark.parametrize("change,text", [
    (dict(dims=(4, 4, 4, 0)), b"extent < 1"),
    (dict(dims=(2048, 2048, 512, 1)), b"too large"),
    (dict(prec_fine=2), b"prec_fine"),
    (dict(prec_coarse=7), b"prec_coarse"),
    (dict(gcr_nkrylov=0), b"solver parameters"),
    (dict(block=[(3, 2, 2, 2)]), b"not divisible by block 3"),
    (dict(nvec=[0]), b"nvec"),
    (dict(nvec=[49]), b"nvec"),
    (dict(link_slots=7), b"link_slots"),
    (dict(prec_fine=1, prec_coarse=2, nvec=[3]), b"even number of null vectors"),
    (dict(prec_fine=1, prec_coarse=0), b"FP64 coarse levels need an FP64 fine level"),
])
def test_create_checks_parameters_before_device_work(lib, change, text):
    """Inconsistent parameters are rejected with MG_ERR_ARG and a message
    before mg_create touches the device (the gauge pointer is never read)."""
    import paper_1612_07873_gb300 as gb
    kw = dict(dims=(4, 4, 4, 4), block=[(2, 2, 2, 2)], nvec=[4])
    kw.update(change)
    p = gb.default_params(**kw)
    h = C.c_void_p()
    assert gb.LIB.mg_create(C.byref(p), C.c_void_p(256), C.byref(h)) == gb.MG_ERR_ARG
    assert text in gb.LIB.mg_last_error(None), gb.LIB.mg_last_error(None)
    assert not h.value


def test_import_without_built_library_raises(tmp_path):
    """No fallback: a copy of the package without its compiled library
    refuses to import."""
    import shutil
    import sys
    pkg = os.path.join(ROOT, "paper_1612_07873_gb300")
    dst = tmp_path / "paper_1612_07873_gb300"
    dst.mkdir()
    for f in os.listdir(pkg):
        if f.endswith(".py"):
            shutil.copy(os.path.join(pkg, f), dst / f)
    code = ("import sys; sys.path.insert(0, %r)\n"
            "try:\n"
            "    import paper_1612_07873_gb300\n"
            "except ImportError as e:\n"
            "    print('refused:', e)\n"
            "else:\n"
            "    print('imported')\n" % str(tmp_path))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, cwd=tmp_path)
    assert r.stdout.startswith("refused:") and "not built" in r.stdout, (r.stdout, r.stderr)


def test_plain_c_program_links_and_calls_the_abi(lib, tmp_path):
    """The library is usable from C without Python: a C99 program compiled
    against include/gbmg.h links libgbmg.so, reads the default parameters
    and gets MG_ERR_ARG with its message for a bad level count (no device
    work happens before that check)."""
    import paper_1612_07873_gb300 as gb
    libdir = os.path.dirname(gb.LIB_PATH)
    src = tmp_path / "abi.c"
    src.write_text(
        '#include <stdio.h>\n#include "gbmg.h"\n'
        "int main(void) {\n"
        "  mg_params p; mg_ctx* ctx = 0; mg_default_params(&p);\n"
        "  p.dims[0] = p.dims[1] = p.dims[2] = p.dims[3] = 4; p.nlevels = 9;\n"
        "  mg_status s = mg_create(&p, (const void*)256, &ctx);\n"
        '  printf("%d %d %s|%s|%s\\n", p.gcr_nkrylov, (int)s, mg_status_string(s),\n'
        '         mg_last_error(0), ctx ? "ctx" : "null");\n'
        "  return s == MG_ERR_ARG ? 0 : 1;\n}\n")
    exe = tmp_path / "abi"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror",
                    "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir, "-lgbmg",
                    f"-Wl,-rpath,{libdir}", "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == "10 -1 invalid argument|mg_create: nlevels must be 2..4|null"
