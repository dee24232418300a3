"""The C-ABI library loads, exports every symbol include/dfmnmf.h declares,
and rejects bad descriptors on the host (no GPU needed for these paths)."""
import os
import re

import numpy as np
import pytest

from paper_2605_19388_gb300 import build as B
from paper_2605_19388_gb300 import dfmnmf as D

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return D.load_library()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "dfmnmf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dfmnmf_[a-z_]+)\s*\(", text)))


def test_header_symbols_exported(lib):
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(D.EXPORTED)


def test_header_constants_match_the_binding():
    """Every enumerator of include/dfmnmf.h has the same value in the Python binding."""
    text = open(os.path.join(ROOT, "include", "dfmnmf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    consts = dict((k, int(v)) for k, v in re.findall(r"\b(DFMNMF_[A-Z0-9_]+)\s*=\s*(\d+)", text))
    assert "DFMNMF_OPT_WAIT_CYCLES" in consts and len(consts) >= 20
    for k, v in consts.items():
        assert getattr(D, k) == v, k


def test_version(lib):
    assert D.dfmnmf_version() == 100


def _args(F=3, T=4, mics=(4, 4), N=2, B_=3):
    M = sum(mics)
    return dict(F=F, T=T, mics=mics, N=N, B=B_, x=np.zeros((F, T, M), np.complex64),
                W0=np.ones((N, F, B_), np.float32), H0=np.ones((N, B_, T), np.float32),
                g0=np.ones((F, N, M), np.float32))


@pytest.mark.parametrize("bad", [dict(F=0), dict(T=0), dict(N=0), dict(B_=0), dict(mics=(4, 3)),
                                 dict(mics=(5,)), dict(mics=(0,)), dict(N=17), dict(B_=65),
                                 dict(mics=(1,) * 17), dict(mics=(16, 16)), dict(mics=(8,)),
                                 dict(mics=(32, 32)), dict(mics=(24,)), dict(mics=(64,))])
def test_invalid_descriptor_rejected(lib, bad):
    a = _args(**bad)
    with pytest.raises(D.DfmnmfError) as ei:
        D.dfmnmf_init(a["F"], a["T"], a["mics"], a["N"], a["B"], a["x"], a["W0"], a["H0"], a["g0"])
    assert ei.value.code == D.DFMNMF_EINVAL


def test_unknown_precision_rejected(lib):
    a = _args()
    for kw in (dict(precision=7), dict(ip_arith=9)):
        with pytest.raises(D.DfmnmfError) as ei:
            D.dfmnmf_init(a["F"], a["T"], a["mics"], a["N"], a["B"], a["x"], a["W0"], a["H0"], a["g0"], **kw)
        assert ei.value.code == D.DFMNMF_EINVAL
    a = _args(mics=(16,))  # the all-microphone block is built in the FP32 form only
    for kw in (dict(precision=D.DFMNMF_BF16_TC),):
        with pytest.raises(D.DfmnmfError) as ei:
            D.dfmnmf_init(a["F"], a["T"], a["mics"], a["N"], a["B"], a["x"], a["W0"], a["H0"], a["g0"], **kw)
        assert ei.value.code == D.DFMNMF_EINVAL


def test_null_arguments_rejected(lib):
    import ctypes
    assert lib.dfmnmf_iterate(None, 1, None) == D.DFMNMF_EINVAL
    assert lib.dfmnmf_loglik(None, None, None) == D.DFMNMF_EINVAL
    assert lib.dfmnmf_run_stage(None, 1, None) == D.DFMNMF_EINVAL
    assert lib.dfmnmf_init(None, None, None, None, None, None, None, None) == D.DFMNMF_EINVAL
    assert b"null" in lib.dfmnmf_last_error()
    assert lib.dfmnmf_autotune(None, 3, None, None, None) == D.DFMNMF_EINVAL
    assert lib.dfmnmf_init_from_images(None, None, None, None) == D.DFMNMF_EINVAL
    assert lib.dfmnmf_batch_create(None, None, 0) == D.DFMNMF_EINVAL
    out = ctypes.c_void_p()
    assert lib.dfmnmf_batch_create(ctypes.byref(out), None, 2) == D.DFMNMF_EINVAL
    assert lib.dfmnmf_batch_iterate(None, 1, None) == D.DFMNMF_EINVAL
    lib.dfmnmf_batch_destroy(None)  # no-op
    lib.dfmnmf_destroy(None)
    assert lib.dfmnmf_launches_per_iteration(None) == -1
    assert lib.dfmnmf_set_option(None, 1, 1) == D.DFMNMF_EINVAL
    assert lib.dfmnmf_get_option(None, 1) == -1


def test_tensor_core_forms_reject_unbuilt_layouts(lib):
    """The tensor-core covariances (bfloat16 or TF32 split operands) are built for M_k = 4 with K in
    {1, 2, 4, 8}; other layouts are rejected before any device work."""
    for mics in ((2, 2), (4, 4, 4), (3, 3)):
        for prec in (D.DFMNMF_BF16_TC, D.DFMNMF_TF32_TC):
            a = _args(mics=mics)
            with pytest.raises(D.DfmnmfError) as ei:
                D.dfmnmf_init(a["F"], a["T"], a["mics"], a["N"], a["B"], a["x"], a["W0"], a["H0"], a["g0"],
                              precision=prec)
            assert ei.value.code == D.DFMNMF_EINVAL, (mics, prec)


def test_noalloc_rejects_sizes_beyond_its_static_scratch(lib):
    """The allocation-free cost keeps F*ceil(T/128) + F*K + 1 partial sums in a
    static array of DFMNMF_NOALLOC_SCRATCH_DOUBLES; larger problems, bad layouts
    and null pointers are refused on the host, before any device call."""
    import ctypes
    dummy = ctypes.c_void_p(1)  # never dereferenced: every case below fails validation first
    out = ctypes.c_double()

    def call(F, T, mics, N=2, B_=3, ptr=dummy):
        m = (ctypes.c_int * len(mics))(*mics)
        d = D.dfmnmf_desc(F, T, len(mics), m, N, B_, 0, 0, 0.0)
        return lib.dfmnmf_loglik_noalloc(ctypes.byref(d), ptr, ptr, ptr, ptr, ptr, ctypes.byref(out), None)

    scratch = 65536
    F = 4000  # 4000 * ceil(2000 / 128) + 4000 * 2 + 1 = 72001 > scratch
    assert F * ((2000 + 127) // 128) + F * 2 + 1 > scratch
    assert call(F, 2000, (4, 4)) == D.DFMNMF_EINVAL
    assert b"exceeds the maximum" in lib.dfmnmf_last_error()
    assert call(3, 20, (4, 3)) == D.DFMNMF_EINVAL      # unequal subarrays
    assert call(3, 20, (4, 4), N=17) == D.DFMNMF_EINVAL
    assert call(0, 20, (4, 4)) == D.DFMNMF_EINVAL
    assert call(3, 20, (4, 4), ptr=None) == D.DFMNMF_EINVAL


def test_noalloc_wrapper_refuses_host_and_wrong_sized_arrays(lib):
    """The binding refuses arrays the library could only read through a host pointer or out of
    bounds: host arrays, and tensors whose element counts do not match the sizes, before any call."""
    torch = pytest.importorskip("torch")
    F, T, mics, N, B_ = 3, 20, (4, 4), 2, 3
    M = sum(mics)
    host = dict(x=np.zeros((F, T, M), np.complex64), Q=np.zeros((F, 32), np.complex128),
                W=np.zeros((N, F, B_), np.float32), H=np.zeros((N, B_, T), np.float32),
                g=np.zeros((F, N, M), np.float32))
    with pytest.raises(ValueError, match="CUDA tensor"):
        D.dfmnmf_loglik_noalloc(F, T, mics, N, B_, **host)
    cpu = {k: torch.from_numpy(v) for k, v in host.items()}
    with pytest.raises(ValueError, match="CUDA tensor"):
        D.dfmnmf_loglik_noalloc(F, T, mics, N, B_, **cpu)
    if torch.cuda.is_available():  # wrong element counts are refused on the GPU machine too
        dev = {k: v.cuda() for k, v in cpu.items()}
        dev["H"] = torch.zeros((N, B_, T - 1), dtype=torch.float32, device="cuda")
        with pytest.raises(ValueError, match="elements"):
            D.dfmnmf_loglik_noalloc(F, T, mics, N, B_, **dev)


CACHE_TEST = r"""
#include <cstdio>
#include "noalloc_cache.h"
int main() {
  dfm::ScratchCache<double*, 4> c;
  double a = 0, b = 0;
  double* out = nullptr;
  if (c.find(7, &out)) return 1;                   // empty table: miss
  if (c.insert(0, &a)) return 2;                   // key 0 ("no context") is never stored
  if (!c.insert(7, &a)) return 3;
  if (!c.find(7, &out) || out != &a) return 4;     // hit
  if (c.find(8, &out)) return 5;                   // another context (a reset device, another
                                                   // context on the same device) misses
  if (!c.insert(8, &b) || !c.find(8, &out) || out != &b) return 6;
  if (!c.find(7, &out) || out != &a) return 7;     // entries never change once stored
  if (!c.insert(9, &a) || !c.insert(10, &a)) return 8;
  if (c.insert(11, &b) || c.find(11, &out)) return 9;  // full: refused, the caller looks up uncached
  std::puts("ok");
  return 0;
}
"""


def test_noalloc_address_cache_is_keyed_by_context(tmp_path):
    """The allocation-free entry point caches the scratch array's device address per CUDA context id
    (not per device number): a new context misses and is looked up anew; stored entries never change;
    a full table stops caching.  Host-only unit test of the cache (compiled with the host compiler)."""
    import shutil
    import subprocess
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "cache_test.cpp"
    src.write_text(CACHE_TEST)
    exe = tmp_path / "cache_test"
    inc = os.path.join(ROOT, "paper_2605_19388_gb300", "csrc")
    subprocess.run([cxx, "-std=c++17", "-O1", "-I", inc, str(src), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip() == "ok", (r.returncode, r.stdout)
