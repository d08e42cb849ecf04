"""Host-side checks of the C ABI: the library loads, exports every declared symbol,
its struct layouts match the binding, and argument validation rejects bad input
before touching a GPU.  No transform is computed here."""

import ctypes as C
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import paper_2505_23618_gb300 as adj
from paper_2505_23618_gb300 import _lib

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "adjtx.h")


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(_lib.LIB_PATH):
        from paper_2505_23618_gb300 import build
        build.build()
    return _lib.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(adj_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_set():
    assert declared_functions() == sorted(_lib.EXPORTED)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", _lib.LIB_PATH], capture_output=True, text=True).stdout
    for name in declared_functions():
        assert re.search(rf"\bT {name}\b", out), f"{name} not exported with C linkage"


def test_struct_layout_matches_c(tmp_path):
    src = tmp_path / "layout.c"
    src.write_text(f"""
#include <stdio.h>
#include <stddef.h>
#include "{HEADER}"
int main(void) {{
  printf("%zu %zu %zu %zu %zu %zu\\n", sizeof(adj_1d_desc_t), offsetof(adj_1d_desc_t, layer_parity),
         offsetof(adj_1d_desc_t, k), offsetof(adj_1d_desc_t, q), sizeof(adj_block_t), sizeof(adj_plan_info_t));
  printf("%d %d %d %d %d %d %d\\n", ADJ_ERR_INVALID_ARG, ADJ_ERR_UNSUPPORTED_SIZE, ADJ_ERR_PARAM_MISMATCH,
         ADJ_ERR_MISALIGNED, ADJ_ERR_CUDA, ADJ_ERR_NO_BLOCKS, ADJ_ERR_NO_MEMORY);
  return 0;
}}""")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", str(src), "-o", str(exe)], check=True)
    sizes, codes = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")[:2]
    assert [int(x) for x in sizes.split()] == [
        C.sizeof(_lib.Adj1dDesc), _lib.Adj1dDesc.layer_parity.offset, _lib.Adj1dDesc.k.offset,
        _lib.Adj1dDesc.q.offset, _lib.BLOCK_DTYPE.itemsize, C.sizeof(_lib.AdjPlanInfo)]
    assert [int(x) for x in codes.split()] == [-1, -2, -3, -4, -5, -6, -7]
    assert sorted(_lib.ERR_CODE.values()) == [-7, -6, -5, -4, -3, -2, -1]


def _create(lib, tfs):
    d = _lib._DescArray(tfs)
    h = C.c_void_p()
    rc = lib.adj_plan_create(C.byref(h), d.arr, d.n, 0)
    return rc, h, lib.adj_last_error().decode()


def _q(k, seed=0):
    Z = np.random.default_rng(seed).standard_normal((k, k))
    return np.linalg.qr(Z)[0]


@pytest.mark.parametrize("tf,code", [
    (dict(n=12, core=0, kind=0), "ADJ_ERR_UNSUPPORTED_SIZE"),
    (dict(n=2, core=0, kind=0), "ADJ_ERR_UNSUPPORTED_SIZE"),
    (dict(n=8, core=4, kind=0), "ADJ_ERR_INVALID_ARG"),
    (dict(n=8, core=0, kind=4), "ADJ_ERR_INVALID_ARG"),
    (dict(n=8, core=0, kind=3, q=_q(4)), "ADJ_ERR_PARAM_MISMATCH"),
    (dict(n=8, core=0, kind=3, q=3 * _q(8)), "ADJ_ERR_PARAM_MISMATCH"),
    (dict(n=8, core=0, kind=2, q=_q(9)), "ADJ_ERR_UNSUPPORTED_SIZE"),
    (dict(n=8, core=0, kind=2, q=2 * _q(4)), "ADJ_ERR_PARAM_MISMATCH"),
    (dict(n=8, core=0, kind=1, parities=np.array([0, 2], np.uint8), angles=np.zeros(7)), "ADJ_ERR_INVALID_ARG"),
    (dict(n=8, core=0, kind=1, parities=np.zeros(65, np.uint8), angles=np.zeros(65 * 4)), "ADJ_ERR_UNSUPPORTED_SIZE"),
    (dict(n=8, core=0, kind=1, parities=np.array([0], np.uint8), angles=np.array([0, 0, np.nan, 0.])),
     "ADJ_ERR_PARAM_MISMATCH"),
])
def test_create_rejects_bad_transforms(lib, tf, code):
    rc, h, msg = _create(lib, [tf])
    assert rc == _lib.ERR_CODE[code], msg
    assert not h.value and msg


def test_create_rejects_null_and_counts(lib):
    h = C.c_void_p()
    assert lib.adj_plan_create(None, None, 0, 0) == _lib.ERR_CODE["ADJ_ERR_INVALID_ARG"]
    assert lib.adj_plan_create(C.byref(h), None, 3, 0) == _lib.ERR_CODE["ADJ_ERR_INVALID_ARG"]
    d = _lib._DescArray([dict(n=8, core=0, kind=0)])
    assert lib.adj_plan_create(C.byref(h), d.arr, 1, 7) == _lib.ERR_CODE["ADJ_ERR_INVALID_ARG"]


def test_null_plan_calls_fail_cleanly(lib):
    for f in ("adj_transform_fwd", "adj_transform_inv", "adj_transform_fwd_f32", "adj_transform_fwd_host",
              "adj_transform_inv_host"):
        assert getattr(lib, f)(None, None, None, None) == _lib.ERR_CODE["ADJ_ERR_INVALID_ARG"]
    assert lib.adj_plan_set_blocks(None, None, 0, 0) == _lib.ERR_CODE["ADJ_ERR_INVALID_ARG"]
    assert lib.adj_plan_prepare_multiple(None, None, None) == _lib.ERR_CODE["ADJ_ERR_INVALID_ARG"]
    assert lib.adj_transform_fwd_multiple(None, None, None, None, None) == _lib.ERR_CODE["ADJ_ERR_INVALID_ARG"]
    lib.adj_plan_destroy(None)


def test_no_cpu_fallback_without_gpu(lib):
    """A valid plan needs a CUDA device: without one the call fails, it never computes on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, h, msg = _create(lib, [dict(n=8, core=0, kind=0)])
    assert rc == _lib.ERR_CODE["ADJ_ERR_CUDA"] and not h.value, msg


def test_generated_cores_are_current():
    import importlib.util
    path = os.path.join(ROOT, "paper_2505_23618_gb300", "csrc", "gen_cores.py")
    spec = importlib.util.spec_from_file_location("gen_cores", path)
    g = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(g)
    text = g.generate()   # raises if a flow graph is off its definition
    with open(os.path.join(os.path.dirname(path), "cores_gen.cuh")) as f:
        assert f.read() == text


_NO_MEMORY_SCRIPT = r"""
import resource
import numpy as np
import synth
import paper_2505_23618_gb300 as adj
from paper_2505_23618_gb300 import _lib
_lib.lib()
n = 1 << 20
blocks = np.zeros(n, dtype=synth.BLOCK_DTYPE)
blocks["w"] = blocks["h"] = 4
blocks["offset"] = np.arange(n) * 16
vm = [int(l.split()[1]) * 1024 for l in open("/proc/self/status") if l.startswith("VmSize")][0]
resource.setrlimit(resource.RLIMIT_AS, (vm + (4 << 20), resource.RLIM_INFINITY))
try:
    adj.layout_preview([synth.Tf(n=4, core=0)], blocks, n * 16)
    print("no error")
except adj.AdjError as e:
    print(e.name)
"""


def test_host_allocation_failure_is_an_error_code():
    """A failed host allocation inside the library comes back as ADJ_ERR_NO_MEMORY, not as a
    C++ exception through the C ABI (which would abort the process).  The planner's tables
    for a million blocks are built under an address-space limit 4 MiB above current use."""
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _NO_MEMORY_SCRIPT], cwd=root, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.strip().splitlines()[-1] == "ADJ_ERR_NO_MEMORY"
