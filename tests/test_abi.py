"""The C ABI library builds, loads and exports what include/sdfdock.h declares (no GPU needed)."""

import ctypes as ct
import os
import re

import numpy as np
import pytest

from paper_1712_00238_gb300 import build as pbuild
from paper_1712_00238_gb300 import sdfdock

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(sd_[a-z0-9_]+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    pbuild.build()
    return sdfdock.load()


def test_exports_every_declared_symbol(lib):
    names = _declared_symbols()
    assert {"sd_create", "sd_sdf_build", "sd_score_rotations", "sd_top_k_poses", "sd_score_grad"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert set(sdfdock._SIGS) >= names


@pytest.mark.parametrize("length", [8, 16, 24, 32, 48, 64, 96, 128, 192, 256, 384, 512])
def test_host_line_fft_matches_dft(lib, length):
    rng = np.random.default_rng(length)
    x = rng.standard_normal(length) + 1j * rng.standard_normal(length)
    a = np.ascontiguousarray(np.stack([x.real, x.imag], 1))
    for inv in (0, 1):
        o = np.zeros_like(a)
        assert lib.sd_host_line_fft(length, inv, a.ctypes.data, o.ctypes.data) == 0
        y = o[:, 0] + 1j * o[:, 1]
        ref = np.fft.ifft(x) * length if inv else np.fft.fft(x)
        assert np.abs(y - ref).max() < 1e-12 * np.abs(ref).max()
    assert lib.sd_host_line_fft(100, 0, a.ctypes.data, a.ctypes.data) == sdfdock.SD_ERR_ARG


def test_defaults_and_argument_errors_without_device(lib):
    p = sdfdock.sd_params()
    assert lib.sd_default_params(ct.byref(p), 3, sdfdock.SD_F32) == 0
    assert (p.lambda1, p.lambda2, p.sigma_t, p.eps, p.w, p.alpha) == (1.0, 3.0, 0.5, 1.5, 6, 2)
    h = ct.c_void_p()
    bad = sdfdock.sd_params()
    lib.sd_default_params(ct.byref(bad), 4, 0)
    assert lib.sd_create(ct.byref(h), 0, ct.byref(bad)) == sdfdock.SD_ERR_ARG
    assert b"dim" in lib.sd_last_error(None)
    lib.sd_default_params(ct.byref(bad), 3, 0)
    bad.w = 9
    assert lib.sd_create(ct.byref(h), 0, ct.byref(bad)) == sdfdock.SD_ERR_ARG
    bad.w = 6
    bad.alpha = 3
    assert lib.sd_create(ct.byref(h), 0, ct.byref(bad)) == sdfdock.SD_ERR_UNIMPLEMENTED
    # NULL contexts are rejected before any CUDA call
    assert lib.sd_sdf_build(None, None, None, None, 1, None, None, 1, None, None, None, None) == sdfdock.SD_ERR_ARG
    assert lib.sd_destroy(None) == 0
    assert lib.sd_shape_free(None) == 0


def test_rotation_sharding_covers_all():
    for n in (1, 7, 576, 54000):
        for world in (1, 2, 3, 8):
            spans = [sdfdock.shard_range(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))


def test_header_is_plain_c(tmp_path):
    # the boundary is a C ABI: the header compiles as strict C99 with every type it declares
    import shutil
    import subprocess

    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "abi.c"
    src.write_text('#include "sdfdock.h"\n'
                   "int main(void) { sd_params p; sd_grid g; sd_cand c; sd_pose o; sd_pair_job j;\n"
                   "  sd_pair_stat s; sd_refine_params r;\n"
                   "  (void)p; (void)g; (void)c; (void)o; (void)j; (void)s; (void)r;\n"
                   "  return SD_OK + SD_F32 + SD_PHI_SDF + SD_REFINE_ASCENT; }\n")
    include = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include")
    r = subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", include,
                        "-fsyntax-only", str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
