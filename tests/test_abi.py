"""The C-ABI library builds, loads and exports every symbol include/ht.h
declares, and the benchmark's probe library those of include/ht_probe.h
(no compute call: this runs without a GPU)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols(header="ht.h"):
    hdr = open(os.path.join(ROOT, "include", header)).read()
    return set(re.findall(r"^(?:ht_status|size_t|int32_t|int64_t|const char \*)\s*\**\s*(ht_\w+)\(",
                          hdr, re.M))


def test_header_declares_the_path():
    syms = declared_symbols()
    for s in ("ht_geometry_create", "ht_geometry_destroy", "ht_vote", "ht_find_peaks",
              "ht_associate", "ht_vote_z", "ht_last_error", "ht_run_event"):
        assert s in syms


def _have_nvcc():
    import shutil
    return os.path.exists("/usr/local/cuda/bin/nvcc") or shutil.which("nvcc") is not None


def test_library_exports_every_declared_symbol():
    from paper_1309_6275_gb300 import build
    if not _have_nvcc():
        pytest.skip("no nvcc on this machine")
    path = build.build()          # a compile or link error fails the test
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (ht_\w+)$", out, re.M))
    missing = declared_symbols() - exported
    assert not missing, f"declared but not exported: {missing}"
    lib = ctypes.CDLL(path)
    for s in declared_symbols():
        assert hasattr(lib, s)
    assert not exported & declared_symbols("ht_probe.h"), "the probe is not part of libht"


def test_probe_library_exports_its_header():
    from paper_1309_6275_gb300 import build
    if not _have_nvcc():
        pytest.skip("no nvcc on this machine")
    path = build.build_probe()
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r"\bT (ht_\w+)$", out, re.M))
    assert declared_symbols("ht_probe.h") == {"ht_probe_shared_atomic_rate"} <= exported


def test_binding_signatures_cover_the_header():
    from paper_1309_6275_gb300 import ht
    assert {n for n, _, _ in ht.SIGNATURES} == declared_symbols()


def test_create_rejects_bad_geometry_without_touching_the_gpu():
    """Argument checks come before any CUDA call."""
    from paper_1309_6275_gb300 import ht
    if not _have_nvcc():
        pytest.skip("no nvcc on this machine")
    lib = ht.lib()
    d = ht._Desc(64, 64, 60, 128, 128, 7, 32, 0, 0.01, 10.0, 32.0, 6.5)   # n_phi0 % 8 != 0
    h = ctypes.c_void_p()
    assert lib.ht_geometry_create(ctypes.byref(d), ctypes.byref(h)) == 1
    assert b"unsupported" in lib.ht_last_error()
    assert lib.ht_geometry_create(None, ctypes.byref(h)) == 1


def test_every_call_rejects_null_arguments_before_any_cuda_call():
    """Failure detection on the host: each status-returning entry point,
    given null handles and pointers and zero sizes, returns HT_ERR_ARG with a
    message naming it (the checks run before any CUDA call, so this needs no
    GPU); the destroy calls accept null as a no-op."""
    from paper_1309_6275_gb300 import ht
    if not _have_nvcc():
        pytest.skip("no nvcc on this machine")
    lib = ht.lib()
    checked = 0
    for name, res, args in ht.SIGNATURES:
        if res is not ht._I32 or name == "ht_mlp_param_count":
            continue
        vals = [0.0 if a in (ctypes.c_float, ctypes.c_double)
                else 0 if a in (ht._I32, ht._SZ, ctypes.c_int64) else None for a in args]
        status = getattr(lib, name)(*vals)
        if name.endswith("_destroy"):
            assert status == 0, name
            continue
        assert status == 1, (name, status)          # HT_ERR_ARG
        assert lib.ht_last_error().decode().startswith(name), (name, lib.ht_last_error())
        checked += 1
    assert checked >= 25


C_PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "ht.h"

int main(void)
{
    /* n_phi0 = 60 is not a multiple of 8: refused before any CUDA call */
    ht_geometry_desc d;
    memset(&d, 0, sizeof d);
    d.n_rho = 64; d.n_d0 = 64; d.n_phi0 = 60; d.n_z0 = 128; d.n_cot = 128;
    d.threshold = 7; d.count_bits = 32;
    d.rho_max = 0.01; d.d0_half = 10.0; d.z0_max = 32.0; d.cot_max = 6.5;
    ht_geometry *g = NULL;
    const ht_status s = ht_geometry_create(&d, &g);
    const ht_status t = ht_vote(NULL, NULL, NULL, 0, NULL, NULL, NULL);
    printf("%d %d %s\n", (int)s, (int)t, ht_last_error());
    return (s == HT_ERR_ARG && t == HT_ERR_ARG && g == NULL) ? 0 : 1;
}
"""


def test_headers_are_plain_c_and_a_c_program_links_and_runs(tmp_path):
    """The boundary is a C ABI: both headers compile as pedantic C11 (and
    C++17), and a C program built against libht.so calls it (argument
    checks only, so no GPU is needed)."""
    import shutil
    from paper_1309_6275_gb300 import build
    if not (_have_nvcc() and shutil.which("gcc") and shutil.which("g++")):
        pytest.skip("no nvcc or gcc on this machine")
    inc = os.path.join(ROOT, "include")
    for name in sorted(os.listdir(inc)):
        if not name.endswith(".h"):
            continue
        for cc, std in (("gcc", "-std=c11"), ("g++", "-std=c++17")):
            src = f'#include "{name}"\nint main(void) {{ return 0; }}\n'
            r = subprocess.run([cc, "-x", "c" if cc == "gcc" else "c++", std, "-Wall", "-Wextra",
                                "-pedantic", "-Werror", "-fsyntax-only", "-I", inc, "-"],
                               input=src, capture_output=True, text=True)
            assert r.returncode == 0, (name, cc, r.stderr)
    lib = build.build()
    cuda_lib = "/usr/local/cuda/lib64"
    (tmp_path / "use_ht.c").write_text(C_PROGRAM)
    exe = str(tmp_path / "use_ht")
    r = subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", inc, str(tmp_path / "use_ht.c"),
                        lib, f"-Wl,-rpath,{os.path.dirname(lib)}", f"-Wl,-rpath-link,{cuda_lib}",
                        "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, LD_LIBRARY_PATH=cuda_lib + ":" + os.environ.get("LD_LIBRARY_PATH", ""))
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=60)
    assert r.returncode == 0, (r.stdout, r.stderr)
    assert r.stdout.startswith("1 1 ht_vote:")
