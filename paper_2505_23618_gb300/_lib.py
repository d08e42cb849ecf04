"""ctypes binding of the C ABI in include/adjtx.h (argument marshalling only).

Every transform runs in the CUDA library; if ``_build/libadjtx.so`` is missing the
import fails loudly (build it with ``python -c "import __graft_entry__ as g; g.build()"``).
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libadjtx.so")

ADJ_OK = 0
ERRORS = {
    -1: "ADJ_ERR_INVALID_ARG",
    -2: "ADJ_ERR_UNSUPPORTED_SIZE",
    -3: "ADJ_ERR_PARAM_MISMATCH",
    -4: "ADJ_ERR_MISALIGNED",
    -5: "ADJ_ERR_CUDA",
    -6: "ADJ_ERR_NO_BLOCKS",
    -7: "ADJ_ERR_NO_MEMORY",
}
ERR_CODE = {v: k for k, v in ERRORS.items()}

EXPORTED = (
    "adj_plan_create", "adj_plan_set_blocks", "adj_plan_update_params",
    "adj_transform_fwd", "adj_transform_inv", "adj_transform_fwd_host",
    "adj_transform_inv_host", "adj_plan_info", "adj_plan_destroy", "adj_last_error",
    "adj_transform_fwd_uniform_noalloc", "adj_transform_fwd_plain", "adj_transform_inv_plain",
    "adj_graph_create", "adj_graph_launch", "adj_graph_destroy", "adj_transform_bwd",
    "adj_plan_param_layout", "adj_coding_gain_proxy", "adj_plan_get_tuning", "adj_plan_set_tuning",
    "adj_plan_autotune", "adj_plan_prepare_multiple", "adj_transform_fwd_multiple",
    "adj_plan_set_frame_blocks", "adj_transform_fwd_frame", "adj_transform_inv_frame",
    "adj_transform_fwd_f32", "adj_layout_preview",
)
DTYPE_INT16, DTYPE_FP32 = 0, 1
GRAPH_FWD, GRAPH_INV, GRAPH_FWD_PLAIN, GRAPH_INV_PLAIN, GRAPH_ROUNDTRIP, GRAPH_FWD_MULTIPLE = range(6)


class Adj1dDesc(C.Structure):
    _fields_ = [("n", C.c_int32), ("core", C.c_int32), ("kind", C.c_int32),
                ("n_layers", C.c_int32), ("layer_parity", C.POINTER(C.c_uint8)),
                ("angles", C.POINTER(C.c_double)), ("k", C.c_int32),
                ("q", C.POINTER(C.c_double))]


class AdjTuning(C.Structure):
    _fields_ = [("cap_div", C.c_int32 * 25), ("ctas_per_sm", C.c_int32), ("ranges_per_sm", C.c_int32),
                ("tail_pct", C.c_int32)]


class AdjPlanInfo(C.Structure):
    _fields_ = [("n_blocks", C.c_int64), ("total_coefs", C.c_int64), ("n_tiles", C.c_int32),
                ("grid_fwd", C.c_int32), ("grid_inv", C.c_int32), ("threads", C.c_int32),
                ("smem_bytes", C.c_int32), ("n_sm", C.c_int32)]


BLOCK_DTYPE = np.dtype([("offset", "<i8"), ("w", "<u2"), ("h", "<u2"),
                        ("tf_h", "<u2"), ("tf_v", "<u2")])
FRAME_BLOCK_DTYPE = np.dtype([("x", "<i4"), ("y", "<i4"), ("w", "<u2"), ("h", "<u2"),
                              ("tf_h", "<u2"), ("tf_v", "<u2")])  # adj_frame_block_t


class AdjError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code
        self.name = ERRORS.get(code, str(code))


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"adjtx CUDA library not built ({path} missing); run the build first")
    lib = C.CDLL(path)
    vp, i32, i64 = C.c_void_p, C.c_int32, C.c_int64
    lib.adj_plan_create.argtypes = [C.POINTER(vp), C.POINTER(Adj1dDesc), i32, i32]
    lib.adj_plan_set_blocks.argtypes = [vp, vp, i64, i64]
    lib.adj_plan_update_params.argtypes = [vp, C.POINTER(Adj1dDesc), i32]
    for f in ("adj_transform_fwd", "adj_transform_inv", "adj_transform_fwd_f32", "adj_transform_fwd_host",
              "adj_transform_inv_host", "adj_transform_fwd_plain", "adj_transform_inv_plain"):
        getattr(lib, f).argtypes = [vp, vp, vp, vp]
    lib.adj_plan_info.argtypes = [vp, C.POINTER(AdjPlanInfo)]
    lib.adj_transform_fwd_uniform_noalloc.argtypes = [C.POINTER(Adj1dDesc), C.POINTER(Adj1dDesc), i64, vp, vp, vp]
    lib.adj_transform_bwd.argtypes = [vp, vp, i32, vp, vp, vp, vp]
    lib.adj_plan_param_layout.argtypes = [vp, C.POINTER(C.c_int32)]
    lib.adj_coding_gain_proxy.argtypes = [vp, i64, i32, vp, vp, vp, vp]
    lib.adj_plan_get_tuning.argtypes = [vp, C.POINTER(AdjTuning)]
    lib.adj_plan_set_tuning.argtypes = [vp, C.POINTER(AdjTuning)]
    lib.adj_plan_autotune.argtypes = [vp, vp, vp, vp, C.c_char_p, i32, vp]
    lib.adj_plan_prepare_multiple.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    lib.adj_transform_fwd_multiple.argtypes = [vp, vp, vp, vp, vp]
    lib.adj_plan_set_frame_blocks.argtypes = [vp, vp, i64, i32, i32, i32]
    lib.adj_transform_fwd_frame.argtypes = [vp, vp, vp, vp]
    lib.adj_transform_inv_frame.argtypes = [vp, vp, vp, vp, vp]
    lib.adj_layout_preview.argtypes = [C.POINTER(Adj1dDesc), i32, vp, i64, i64, i32, vp, vp, i64,
                                       C.POINTER(C.c_int64), vp, i64, C.POINTER(C.c_int64), vp, i32,
                                       C.POINTER(C.c_int32)]
    lib.adj_graph_create.argtypes = [vp, i32, vp, vp, vp, C.POINTER(vp)]
    lib.adj_graph_launch.argtypes = [vp, vp]
    lib.adj_graph_destroy.argtypes = [vp]
    lib.adj_graph_destroy.restype = None
    lib.adj_plan_destroy.argtypes = [vp]
    lib.adj_plan_destroy.restype = None
    lib.adj_last_error.restype = C.c_char_p
    for f in EXPORTED:
        if f not in ("adj_plan_destroy", "adj_last_error", "adj_graph_destroy"):
            getattr(lib, f).restype = C.c_int
    return lib


_lib = None


def lib() -> C.CDLL:
    global _lib
    if _lib is None:
        _lib = load()
    return _lib


def check(rc: int):
    if rc != ADJ_OK:
        raise AdjError(rc, lib().adj_last_error().decode())


def _get(tf, name, default=None):
    if isinstance(tf, dict):
        return tf.get(name, default)
    return getattr(tf, name, default)


class _DescArray:
    """Keeps the numpy buffers referenced by an array of Adj1dDesc alive."""

    def __init__(self, tfs):
        self.keep = []
        self.arr = (Adj1dDesc * max(1, len(tfs)))()
        for i, tf in enumerate(tfs):
            d = self.arr[i]
            d.n, d.core, d.kind = int(_get(tf, "n")), int(_get(tf, "core")), int(_get(tf, "kind", 0))
            par = np.ascontiguousarray(_get(tf, "parities", np.zeros(0)), dtype=np.uint8)
            ang = np.ascontiguousarray(_get(tf, "angles", np.zeros(0)), dtype=np.float64)
            q = _get(tf, "q", None)
            if d.kind == 1:
                d.n_layers = par.size
                d.layer_parity = par.ctypes.data_as(C.POINTER(C.c_uint8))
                d.angles = ang.ctypes.data_as(C.POINTER(C.c_double))
                self.keep += [par, ang]
            if d.kind in (2, 3) and q is not None:
                qa = np.ascontiguousarray(q, dtype=np.float64)
                d.k = qa.shape[0]
                d.q = qa.ctypes.data_as(C.POINTER(C.c_double))
                self.keep.append(qa)
        self.n = len(tfs)


def _ptr(x) -> int:
    """Address of a torch tensor / numpy array / int."""
    if x is None:
        return 0
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return int(x.data_ptr())
    if isinstance(x, np.ndarray):
        return int(x.ctypes.data)
    raise TypeError(f"cannot take the address of {type(x)}")


def _stream(s) -> int:
    if s is None:
        return 0
    if isinstance(s, int):
        return s
    return int(getattr(s, "cuda_stream", s))


class Plan:
    """An adj_plan_t: 1-D transform table + block list, with fwd/inv entry points."""

    def __init__(self, tfs, flags: int = 0):
        self._lib = lib()
        self.tfs = list(tfs)
        self._h = C.c_void_p()
        d = _DescArray(self.tfs)
        check(self._lib.adj_plan_create(C.byref(self._h), d.arr, d.n, flags))
        self.total = 0
        self.n_blocks = 0

    def set_blocks(self, blocks: np.ndarray, total: int):
        b = np.ascontiguousarray(blocks).view(BLOCK_DTYPE)
        check(self._lib.adj_plan_set_blocks(self._h, b.ctypes.data if b.size else None,
                                            b.size, int(total)))
        self.total = int(total)
        self.n_blocks = int(b.size)
        return self

    def update_params(self, tfs):
        d = _DescArray(list(tfs))
        check(self._lib.adj_plan_update_params(self._h, d.arr, d.n))
        self.tfs = list(tfs)

    def fwd(self, d_in, d_out, stream=None):
        check(self._lib.adj_transform_fwd(self._h, _ptr(d_in), _ptr(d_out), _stream(stream)))

    def inv(self, d_in, d_out, stream=None):
        check(self._lib.adj_transform_inv(self._h, _ptr(d_in), _ptr(d_out), _stream(stream)))

    def fwd_f32(self, d_in, d_out, stream=None):
        """Forward of FP32 blocks (adj_transform_fwd_f32)."""
        check(self._lib.adj_transform_fwd_f32(self._h, _ptr(d_in), _ptr(d_out), _stream(stream)))

    def set_frame_blocks(self, blocks: np.ndarray, frame_w: int, frame_h: int, stride: int):
        """Blocks inside a frame (FRAME_BLOCK_DTYPE records); coefficients are packed in list order."""
        b = np.ascontiguousarray(blocks).view(FRAME_BLOCK_DTYPE)
        check(self._lib.adj_plan_set_frame_blocks(self._h, b.ctypes.data if b.size else None, b.size,
                                                  int(frame_w), int(frame_h), int(stride)))
        self.n_blocks = int(b.size)
        self.total = int(np.sum(b["w"].astype(np.int64) * b["h"])) if b.size else 0
        return self

    def fwd_frame(self, d_frame, d_coef, stream=None):
        check(self._lib.adj_transform_fwd_frame(self._h, _ptr(d_frame), _ptr(d_coef), _stream(stream)))

    def inv_frame(self, d_coef, d_frame_f32=None, d_frame_i16=None, stream=None):
        check(self._lib.adj_transform_inv_frame(self._h, _ptr(d_coef), _ptr(d_frame_f32), _ptr(d_frame_i16),
                                                _stream(stream)))

    def prepare_multiple(self):
        """Validate the block list for the Multiple forward; returns the side offsets in
        floats (n_blocks + 1 entries, block list order; the last is the total)."""
        off = np.zeros(self.n_blocks + 1, dtype=np.int64)
        total = C.c_int64()
        check(self._lib.adj_plan_prepare_multiple(self._h, off.ctypes.data_as(C.POINTER(C.c_int64)),
                                                  C.byref(total)))
        return off

    def fwd_multiple(self, d_in, d_coef, d_side, stream=None):
        """2-D DCT-2 into d_coef and the distinct DST-7 / DCT-8 adjusted coefficients of the
        four pairings into d_side (see adj_transform_fwd_multiple)."""
        check(self._lib.adj_transform_fwd_multiple(self._h, _ptr(d_in), _ptr(d_coef), _ptr(d_side),
                                                   _stream(stream)))

    def fwd_plain(self, d_in, d_out, stream=None):
        check(self._lib.adj_transform_fwd_plain(self._h, _ptr(d_in), _ptr(d_out), _stream(stream)))

    def inv_plain(self, d_in, d_out, stream=None):
        check(self._lib.adj_transform_inv_plain(self._h, _ptr(d_in), _ptr(d_out), _stream(stream)))

    def fwd_host(self, h_in, h_out, stream=None):
        check(self._lib.adj_transform_fwd_host(self._h, _ptr(h_in), _ptr(h_out), _stream(stream)))

    def inv_host(self, h_in, h_out, stream=None):
        check(self._lib.adj_transform_inv_host(self._h, _ptr(h_in), _ptr(h_out), _stream(stream)))

    def bwd(self, d_x, d_gy, d_gx=None, d_gparams=None, stream=None, x_fp32=None):
        """Gradients of the forward transform (see adj_transform_bwd)."""
        if x_fp32 is None:
            x_fp32 = getattr(d_x, "dtype", None) is not None and "float" in str(d_x.dtype)
        check(self._lib.adj_transform_bwd(self._h, _ptr(d_x), DTYPE_FP32 if x_fp32 else DTYPE_INT16,
                                          _ptr(d_gy), _ptr(d_gx), _ptr(d_gparams), _stream(stream)))

    def tuning(self) -> dict:
        t = AdjTuning()
        check(self._lib.adj_plan_get_tuning(self._h, C.byref(t)))
        return {"cap_div": list(t.cap_div), "ctas_per_sm": t.ctas_per_sm, "ranges_per_sm": t.ranges_per_sm,
                "tail_pct": t.tail_pct}

    def set_tuning(self, tuning: dict):
        t = AdjTuning()
        t.cap_div[:] = list(tuning["cap_div"])
        t.ctas_per_sm = int(tuning["ctas_per_sm"])
        t.ranges_per_sm = int(tuning["ranges_per_sm"])
        t.tail_pct = int(tuning.get("tail_pct", self.tuning()["tail_pct"]))
        check(self._lib.adj_plan_set_tuning(self._h, C.byref(t)))

    def autotune(self, d_in, d_coef, d_recon, cache_path=None, max_evals=0, stream=None):
        """Time candidate tunings on this plan's blocks and keep the fastest (see the header)."""
        path = cache_path.encode() if cache_path else None
        check(self._lib.adj_plan_autotune(self._h, _ptr(d_in), _ptr(d_coef), _ptr(d_recon), path,
                                          int(max_evals), _stream(stream)))
        return self.tuning()

    def param_layout(self):
        """Offsets of each transform's gradient entries (n_tfs + 1 values)."""
        off = (C.c_int32 * (len(self.tfs) + 1))()
        check(self._lib.adj_plan_param_layout(self._h, off))
        return list(off)

    def graph(self, what, d_in, d_out, d_out2=None):
        """Capture the selected launches for these buffers; returns a Graph."""
        return Graph(self, what, d_in, d_out, d_out2)

    def info(self) -> dict:
        i = AdjPlanInfo()
        check(self._lib.adj_plan_info(self._h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in AdjPlanInfo._fields_}

    def close(self):
        if self._h:
            self._lib.adj_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


class Graph:
    """An adj_graph_t: captured launches of a plan for fixed buffers."""

    def __init__(self, plan, what, d_in, d_out, d_out2=None):
        self._lib = plan._lib
        self.plan = plan            # keeps the plan alive while the graph exists
        self._h = C.c_void_p()
        check(self._lib.adj_graph_create(plan._h, int(what), _ptr(d_in), _ptr(d_out), _ptr(d_out2),
                                         C.byref(self._h)))

    def launch(self, stream=None):
        check(self._lib.adj_graph_launch(self._h, _stream(stream)))

    def close(self):
        if self._h:
            self._lib.adj_graph_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TILE_INFO_DTYPE = np.dtype([("list_begin", "<u4"), ("nblk", "<u2"), ("w", "<u2"), ("h", "<u2"),
                            ("tf_h", "<u2"), ("tf_v", "<u2"), ("pad", "<u2")])


def layout_preview(tfs, blocks: np.ndarray, total: int, n_sm: int = 152) -> dict:
    """The tile and range layout adj_plan_set_blocks would build for a GPU of n_sm SMs, computed
    on the host (adj_layout_preview; no device needed): tiles (TILE_INFO_DTYPE) in launch order,
    their estimated costs, the block-offset list and the range starts."""
    L = lib()
    d = _DescArray(list(tfs))
    b = np.ascontiguousarray(blocks, dtype=BLOCK_DTYPE)
    nt, nl, nr = C.c_int64(0), C.c_int64(0), C.c_int32(0)
    args = (d.arr, d.n, _ptr(b) if b.size else None, int(b.size), int(total), int(n_sm))
    check(L.adj_layout_preview(*args, None, None, 0, C.byref(nt), None, 0, C.byref(nl), None, 0, C.byref(nr)))
    tiles = np.zeros(nt.value, dtype=TILE_INFO_DTYPE)
    costs = np.zeros(nt.value, dtype=np.float64)
    lst = np.zeros(max(1, nl.value), dtype=np.uint32)
    rbeg = np.zeros(nr.value + 1, dtype=np.uint32)
    check(L.adj_layout_preview(*args, _ptr(tiles) if tiles.size else None, _ptr(costs) if costs.size else None,
                               int(nt.value), C.byref(nt), _ptr(lst), int(lst.size), C.byref(nl), _ptr(rbeg),
                               int(nr.value), C.byref(nr)))
    return {"tiles": tiles, "costs": costs, "list": lst[:nl.value], "range_begin": rbeg}
