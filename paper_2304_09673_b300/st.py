"""Thin ctypes binding of ``libst.so`` (include/st.h): argument marshalling only.

Every function keeps the C name.  Device buffers are torch CUDA tensors
passed by pointer; streams are torch streams (default: the current one).
Importing this module loads ``libst.so`` and raises if it is missing: there is
no fallback path.
"""
from __future__ import annotations

import ctypes as C
from pathlib import Path

import numpy as np

LIB_PATH = Path(__file__).resolve().parent / "libst.so"
if not LIB_PATH.exists():
    raise ImportError(f"{LIB_PATH} is missing: build it with python -m paper_2304_09673_b300.build "
                      "(or __graft_entry__.build())")
_lib = C.CDLL(str(LIB_PATH))

ST_OK, ST_ERR_INVALID, ST_ERR_CAPACITY, ST_ERR_CUDA, ST_ERR_TIMEOUT, ST_ERR_NOMEM = 0, -1, -2, -3, -4, -5
ST_STEP_PLAIN, ST_STEP_LEARNED, ST_STEP_OVERRELAX, ST_STEP_CROSSING = 0, 1, 2, 3
ST_TRAVERSE_PARENT, ST_TRAVERSE_FAST = 0, 1
ST_NUM_COUNTERS = 10
ST_REC_FLOATS = 16


class StError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.st_last_error().decode(errors="replace")
        super().__init__(f"{where} failed ({code}): {msg}")
        self.code = code


class st_scene_desc(C.Structure):
    _fields_ = [("n_nodes", C.c_int32), ("root", C.c_int32), ("kind", C.c_void_p),
                ("left", C.c_void_p), ("right", C.c_void_p), ("params", C.c_void_p),
                ("voi_pad", C.c_float)]


class st_camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("target", C.c_float * 3), ("up", C.c_float * 3),
                ("vfov_deg", C.c_float), ("width", C.c_int32), ("height", C.c_int32)]


class st_tiles(C.Structure):
    _fields_ = [("tile", C.c_int32), ("tiles_x", C.c_int32), ("tiles_y", C.c_int32),
                ("offsets", C.c_void_p), ("z_in", C.c_void_p), ("z_out", C.c_void_p),
                ("prim", C.c_void_p), ("n_entries", C.c_uint64), ("max_overlap", C.c_uint32)]


class st_trace_opts(C.Structure):
    _fields_ = [("eps", C.c_float), ("lipschitz", C.c_float), ("max_steps", C.c_int32),
                ("step_mode", C.c_int32), ("depth_slab_frac", C.c_float),
                ("max_new_per_turn", C.c_int32), ("newton_iters", C.c_int32),
                ("newton_clamp", C.c_float), ("mlp", C.c_void_p), ("tile_stats", C.c_void_p),
                ("omega", C.c_float), ("min_step", C.c_float), ("split_kcycles", C.c_int32),
                ("heavy_split_len", C.c_int32), ("heavy_split_rank", C.c_int32), ("wait_spin_limit", C.c_uint32),
                ("check_status", C.c_int32), ("cta_eval_min_view", C.c_int32), ("full_views", C.c_int32)]


class st_tune(C.Structure):
    _fields_ = [("tile", C.c_int32), ("max_new_per_turn", C.c_int32), ("depth_slab_frac", C.c_float),
                ("ms", C.c_float)]


_P = C.c_void_p
_lib.st_last_error.restype = C.c_char_p
_lib.st_version.restype = C.c_char_p
_lib.st_scene_create.argtypes = [C.POINTER(st_scene_desc), C.POINTER(C.c_void_p), _P]
_lib.st_scene_update_prims.argtypes = [_P, _P, _P, C.c_int, _P]
_lib.st_scene_addresses.argtypes = [_P, _P]
_lib.st_scene_info.argtypes = [_P, _P]
_lib.st_scene_destroy.argtypes = [_P]
_lib.st_scene_destroy.restype = None
_lib.st_build_tiles.argtypes = [_P, C.POINTER(st_camera), C.c_int, C.POINTER(st_tiles), _P]
_lib.st_trace.argtypes = [_P, C.POINTER(st_camera), C.POINTER(st_tiles), C.POINTER(st_trace_opts),
                          _P, _P, _P, _P, _P, _P]
_lib.st_tiles_copy.argtypes = [C.POINTER(st_tiles), _P, _P, _P, _P, _P]
_lib.st_pruned_view.argtypes = [_P, _P, C.c_int, _P, _P, _P, _P]
_lib.st_pruned_view_alg1.argtypes = [_P, _P, C.c_int, _P, _P, _P, _P]
_lib.st_pruned_view_live.argtypes = [_P, _P, C.c_int, _P, _P, _P, _P]
_lib.st_eval_pruned.argtypes = [_P, _P, _P, _P, C.c_int, _P, _P, _P]
_lib.st_eval_pruned_levels.argtypes = [_P, _P, C.c_int, _P, _P, _P, C.c_int, _P, _P]
_lib.st_kernel_launches.restype = C.c_uint64
_lib.st_trace_noalloc.argtypes = [_P, C.POINTER(st_camera), C.POINTER(st_tiles), C.POINTER(st_trace_opts),
                                  _P, _P, _P, _P, _P, _P]
_lib.st_trace_noalloc_scratch_bytes.restype = C.c_size_t
_lib.st_trace_noalloc_last_layout.argtypes = [_P]
_lib.st_device_allocations.restype = C.c_uint64
_lib.st_trace_record.argtypes = [_P, C.POINTER(st_camera), C.POINTER(st_tiles), C.POINTER(st_trace_opts),
                                 _P, _P, _P, _P, _P, C.c_uint32, _P, C.c_int, _P]
_lib.st_mlp_pack_size.restype = C.c_size_t
_lib.st_mlp_pack.argtypes = [_P, _P]
_lib.st_mlp_grad.argtypes = [_P, _P, _P, C.c_int, _P, _P, _P]
_lib.st_mlp_grad_bf16.argtypes = [_P, _P, _P, C.c_int, _P, _P, _P]
_lib.st_mlp_adam.argtypes = [_P, _P, _P, _P, C.c_int, C.c_float, C.c_float, C.c_float, C.c_float, C.c_float, _P]
_lib.st_mlp_infer.argtypes = [_P, _P, C.c_int, _P, _P]
_lib.st_prep_tree.argtypes = [C.POINTER(st_scene_desc), _P, _P, _P, _P]
_lib.st_tune_key.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_char_p, C.c_int]
_lib.st_tune_load.argtypes = [C.c_char_p, C.c_char_p, C.POINTER(st_tune)]
_lib.st_tune_store.argtypes = [C.c_char_p, C.c_char_p, C.POINTER(st_tune)]
_lib.st_autotune.argtypes = [_P, C.POINTER(st_camera), C.POINTER(st_trace_opts), C.c_char_p, C.POINTER(st_tune), _P]
_lib.st_batch_create.argtypes = [_P, _P, C.c_int, C.POINTER(st_trace_opts), _P, _P, _P, _P, C.c_char_p,
                                 C.POINTER(C.c_void_p), _P]
_lib.st_batch_render.argtypes = [_P, _P]
_lib.st_batch_tiles.argtypes = [_P, C.c_int]
_lib.st_batch_graph_kernels.argtypes = [_P]
_lib.st_batch_destroy.argtypes = [_P]
_lib.st_batch_destroy.restype = None
_lib.st_render_batch.argtypes = [_P, _P, C.c_int, C.POINTER(st_trace_opts), _P, _P, _P, _P, C.c_char_p, _P]
_lib.st_build_dexels.argtypes = [_P, C.POINTER(st_camera), C.POINTER(st_tiles), C.POINTER(st_tiles), _P]
_lib.st_trace_dexels.argtypes = [_P, C.POINTER(st_camera), C.POINTER(st_tiles), C.POINTER(st_trace_opts), C.c_int,
                                 _P, _P, _P, _P, _P, _P]
_lib.st_eval_sparse.argtypes = [_P, _P, C.c_int, _P, C.c_int, C.c_int, _P, _P, _P]

EXPORTED = ("st_scene_create", "st_scene_update_prims", "st_scene_addresses", "st_scene_info", "st_scene_destroy",
            "st_build_tiles", "st_trace", "st_tiles_copy", "st_pruned_view", "st_pruned_view_alg1", "st_eval_pruned",
            "st_eval_pruned_levels",
            "st_prep_tree", "st_last_error", "st_version", "st_kernel_launches", "st_device_allocations",
            "st_trace_noalloc", "st_trace_noalloc_scratch_bytes", "st_trace_noalloc_last_layout",
            "st_trace_record", "st_mlp_pack_size", "st_mlp_param_count", "st_mlp_pack", "st_mlp_grad",
            "st_mlp_grad_bf16", "st_mlp_adam", "st_mlp_infer", "st_tune_key", "st_tune_load", "st_tune_store", "st_autotune",
            "st_batch_create", "st_batch_render", "st_batch_tiles", "st_batch_graph_kernels", "st_batch_destroy",
            "st_render_batch", "st_build_dexels", "st_trace_dexels", "st_eval_sparse")


def lib():
    return _lib


def _check(rc: int, where: str) -> int:
    if rc < 0:
        raise StError(rc, where)
    return rc


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def make_desc(scene, voi_pad: float = 0.0):
    """st_scene_desc over a scenegen.Scene (the numpy arrays are kept alive
    on the returned object)."""
    kind = np.ascontiguousarray(scene.kind, np.int32)
    left = np.ascontiguousarray(scene.left, np.int32)
    right = np.ascontiguousarray(scene.right, np.int32)
    params = np.ascontiguousarray(scene.params, np.float32)
    d = st_scene_desc(scene.n_nodes, scene.root, kind.ctypes.data, left.ctypes.data,
                      right.ctypes.data, params.ctypes.data, voi_pad)
    d._keep = (kind, left, right, params)
    return d


def make_camera(cam) -> st_camera:
    c = st_camera()
    c.eye[:] = [float(x) for x in cam.eye]
    c.target[:] = [float(x) for x in cam.target]
    c.up[:] = [float(x) for x in cam.up]
    c.vfov_deg = float(cam.vfov_deg)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def make_opts(eps=1e-4, lipschitz=1.45, max_steps=256, step_mode=ST_STEP_PLAIN, depth_slab_frac=0.05,
              max_new_per_turn=32, newton_iters=2, newton_clamp=0.0, mlp=None, tile_stats=None,
              omega=1.7, min_step=0.0, split_kcycles=0, heavy_split_len=0, heavy_split_rank=0, wait_spin_limit=0,
              check_status=0, cta_eval_min_view=0, full_views=0) -> st_trace_opts:
    o = st_trace_opts(eps, lipschitz, max_steps, step_mode, depth_slab_frac, max_new_per_turn,
                      newton_iters, newton_clamp, mlp, None, omega, min_step, split_kcycles,
                      heavy_split_len, heavy_split_rank, wait_spin_limit, check_status, cta_eval_min_view,
                      full_views)
    if tile_stats is not None:
        o.tile_stats = tile_stats.data_ptr()
        o._keep = tile_stats
    return o


# ---- entry points (same names as the C ABI) ----------------------------------------
def st_scene_create(scene, voi_pad: float = 0.0, stream=None) -> C.c_void_p:
    desc = make_desc(scene, voi_pad)
    h = C.c_void_p()
    _check(_lib.st_scene_create(C.byref(desc), C.byref(h), _stream(stream)), "st_scene_create")
    return h


def st_scene_update_prims(h, ids, params, stream=None) -> None:
    ids = np.ascontiguousarray(ids, np.int32)
    params = np.ascontiguousarray(params, np.float32).reshape(len(ids), ST_REC_FLOATS)
    _check(_lib.st_scene_update_prims(h, ids.ctypes.data, params.ctypes.data, len(ids), _stream(stream)),
           "st_scene_update_prims")


def st_scene_addresses(h, n_nodes: int) -> np.ndarray:
    out = np.empty(n_nodes, np.int32)
    _check(_lib.st_scene_addresses(h, out.ctypes.data), "st_scene_addresses")
    return out


def st_scene_info(h) -> dict:
    out = np.zeros(4, np.float64)
    _check(_lib.st_scene_info(h, out.ctypes.data), "st_scene_info")
    return dict(diameter=float(out[0]), extent=float(out[1]), n_prims=int(out[2]), stack_depth=int(out[3]))


def st_scene_destroy(h) -> None:
    _lib.st_scene_destroy(h)


def st_build_tiles(h, cam, tile: int = 16, stream=None) -> st_tiles:
    t = st_tiles()
    c = make_camera(cam)
    _check(_lib.st_build_tiles(h, C.byref(c), tile, C.byref(t), _stream(stream)), "st_build_tiles")
    return t


def st_trace(h, cam, tiles: st_tiles, opts: st_trace_opts | None, depth, normal, evals, flags,
             counters=None, stream=None) -> None:
    c = make_camera(cam)
    o = opts if opts is not None else make_opts()
    _check(_lib.st_trace(h, C.byref(c), C.byref(tiles), C.byref(o), _ptr(depth), _ptr(normal), _ptr(evals),
                         _ptr(flags), _ptr(counters), _stream(stream)), "st_trace")


def st_trace_noalloc(h, cam, tiles: st_tiles, opts: st_trace_opts | None, depth, normal, evals, flags,
                     counters=None, stream=None) -> None:
    """st_trace without device allocation (fixed scratch array in the library)."""
    c = make_camera(cam)
    o = opts if opts is not None else make_opts()
    _check(_lib.st_trace_noalloc(h, C.byref(c), C.byref(tiles), C.byref(o), _ptr(depth), _ptr(normal),
                                 _ptr(evals), _ptr(flags), _ptr(counters), _stream(stream)), "st_trace_noalloc")


def st_trace_noalloc_scratch_bytes() -> int:
    return int(_lib.st_trace_noalloc_scratch_bytes())


def st_trace_noalloc_last_layout() -> dict:
    out = np.zeros(3, np.uint64)
    _check(_lib.st_trace_noalloc_last_layout(out.ctypes.data), "st_trace_noalloc_last_layout")
    return dict(work_in_scratch=bool(out[0]), bytes_used=int(out[1]), split_records=int(out[2]))


def st_device_allocations() -> int:
    return int(_lib.st_device_allocations())


def st_trace_record(h, cam, tiles: st_tiles, opts, depth, normal, evals, flags, records, rec_count,
                    ray_stride: int = 1, stream=None) -> None:
    """Plain tracing that also writes training records (device float[cap][8])."""
    c = make_camera(cam)
    o = opts if opts is not None else make_opts()
    _check(_lib.st_trace_record(h, C.byref(c), C.byref(tiles), C.byref(o), _ptr(depth), _ptr(normal), _ptr(evals),
                                _ptr(flags), _ptr(records), int(records.numel() // 8), _ptr(rec_count), ray_stride,
                                _stream(stream)), "st_trace_record")


MLP_PARAMS = 1313


def st_mlp_pack_size() -> int:
    return int(_lib.st_mlp_pack_size())


def st_mlp_param_count() -> int:
    return int(_lib.st_mlp_param_count())


def st_mlp_pack(params) -> np.ndarray:
    """FP32 parameter vector -> packed bytes (host numpy uint8)."""
    p = np.ascontiguousarray(params, np.float32).reshape(-1)
    if p.size != MLP_PARAMS:
        raise ValueError("expected %d parameters" % MLP_PARAMS)
    out = np.zeros(st_mlp_pack_size(), np.uint8)
    _check(_lib.st_mlp_pack(p.ctypes.data, out.ctypes.data), "st_mlp_pack")
    return out


def st_mlp_grad(params, x, y, grad, loss_sum, stream=None) -> None:
    _check(_lib.st_mlp_grad(_ptr(params), _ptr(x), _ptr(y), int(y.numel()), _ptr(grad), _ptr(loss_sum),
                            _stream(stream)), "st_mlp_grad")


def st_mlp_grad_bf16(params, x, y, grad, loss_sum, stream=None) -> None:
    _check(_lib.st_mlp_grad_bf16(_ptr(params), _ptr(x), _ptr(y), int(y.numel()), _ptr(grad), _ptr(loss_sum),
                                 _stream(stream)), "st_mlp_grad_bf16")


def st_mlp_adam(params, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8, grad_scale=1.0,
                stream=None) -> None:
    _check(_lib.st_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), step, lr, beta1, beta2, eps, grad_scale,
                            _stream(stream)), "st_mlp_adam")


def st_mlp_infer(packed, x, omega, stream=None) -> None:
    _check(_lib.st_mlp_infer(_ptr(packed), _ptr(x), int(omega.numel()), _ptr(omega), _stream(stream)),
           "st_mlp_infer")


def st_pruned_view(h, act, view, view_addr, info, stream=None) -> None:
    _check(_lib.st_pruned_view(h, _ptr(act), int(act.numel()), _ptr(view), _ptr(view_addr), _ptr(info),
                               _stream(stream)), "st_pruned_view")


def st_pruned_view_alg1(h, act, view, view_addr, info, stream=None) -> None:
    _check(_lib.st_pruned_view_alg1(h, _ptr(act), int(act.numel()), _ptr(view), _ptr(view_addr), _ptr(info),
                                    _stream(stream)), "st_pruned_view_alg1")


def st_pruned_view_live(h, act, view, view_addr, info, stream=None) -> None:
    _check(_lib.st_pruned_view_live(h, _ptr(act), int(act.numel()), _ptr(view), _ptr(view_addr), _ptr(info),
                                    _stream(stream)), "st_pruned_view_live")


def st_eval_pruned(h, view, info, pts, f, grad=None, stream=None) -> None:
    _check(_lib.st_eval_pruned(h, _ptr(view), _ptr(info), _ptr(pts), int(pts.numel() // 3), _ptr(f), _ptr(grad),
                               _stream(stream)), "st_eval_pruned")


def st_eval_pruned_levels(h, act, view, info, pts, f, stream=None) -> None:
    _check(_lib.st_eval_pruned_levels(h, _ptr(act), int(act.numel()), _ptr(view), _ptr(info), _ptr(pts),
                                      int(pts.numel() // 3), _ptr(f), _stream(stream)), "st_eval_pruned_levels")


def st_build_dexels(h, cam, tiles: st_tiles, stream=None) -> st_tiles:
    """Full-resolution A-buffer (one list per pixel) from tile lists of the same camera."""
    out = st_tiles()
    c = make_camera(cam)
    _check(_lib.st_build_dexels(h, C.byref(c), C.byref(tiles), C.byref(out), _stream(stream)), "st_build_dexels")
    return out


def st_trace_dexels(h, cam, dexels: st_tiles, opts: st_trace_opts | None, traversal: int, depth, normal, evals,
                    flags, counters=None, stream=None) -> None:
    c = make_camera(cam)
    o = opts if opts is not None else make_opts()
    _check(_lib.st_trace_dexels(h, C.byref(c), C.byref(dexels), C.byref(o), int(traversal), _ptr(depth),
                                _ptr(normal), _ptr(evals), _ptr(flags), _ptr(counters), _stream(stream)),
           "st_trace_dexels")


def st_eval_sparse(h, act, pts, traversal: int, f, status, stream=None) -> None:
    _check(_lib.st_eval_sparse(h, _ptr(act), int(act.numel()), _ptr(pts), int(pts.numel() // 3), int(traversal),
                               _ptr(f), _ptr(status), _stream(stream)), "st_eval_sparse")


def st_tiles_copy(tiles: st_tiles, stream=None):
    """A-buffer to host numpy arrays: (offsets, z_in, z_out, prim)."""
    nt = tiles.tiles_x * tiles.tiles_y + 1
    ne = int(tiles.n_entries)
    off = np.empty(nt, np.uint32)
    zi = np.empty(max(ne, 1), np.float32)
    zo = np.empty(max(ne, 1), np.float32)
    pr = np.empty(max(ne, 1), np.uint32)
    _check(_lib.st_tiles_copy(C.byref(tiles), off.ctypes.data, zi.ctypes.data, zo.ctypes.data,
                              pr.ctypes.data, _stream(stream)), "st_tiles_copy")
    return off, zi[:ne], zo[:ne], pr[:ne]


def st_prep_tree(scene) -> dict:
    """Host-only preparation (no GPU): post-order, packed blobs, parents, ROI."""
    desc = make_desc(scene)
    n = scene.n_nodes
    po = np.empty(n, np.int32)
    blob = np.empty(n, np.uint32)
    parent = np.empty(n, np.int32)
    roi = np.empty(n, np.float32)
    depth = _check(_lib.st_prep_tree(C.byref(desc), po.ctypes.data, blob.ctypes.data, parent.ctypes.data,
                                     roi.ctypes.data), "st_prep_tree")
    return dict(po_of_desc=po, blob=blob, parent=parent, roi=roi, stack_depth=int(depth))


def st_kernel_launches() -> int:
    return int(_lib.st_kernel_launches())


def st_version() -> str:
    return _lib.st_version().decode()


# ---- convenience ----------------------------------------------------------------
class Renderer:
    """One scene on the current CUDA device: owns the st_scene handle and the
    output tensors of one resolution."""

    def __init__(self, scene, cam, tile: int = 16, voi_pad: float = 0.0, stream=None):
        import torch
        self.scene = scene
        self.cam = cam
        self.tile = tile
        self.stream = stream
        self.h = st_scene_create(scene, voi_pad, stream)
        W, H = cam.width, cam.height
        dev = torch.device("cuda")
        self.depth = torch.empty(H * W, dtype=torch.float32, device=dev)
        self.normal = torch.empty(H * W * 3, dtype=torch.float32, device=dev)
        self.evals = torch.empty(H * W, dtype=torch.int32, device=dev)
        self.flags = torch.empty(H * W, dtype=torch.uint8, device=dev)
        self.counters = torch.zeros(ST_NUM_COUNTERS, dtype=torch.int64, device=dev)
        self.tiles = None

    def build_tiles(self):
        self.tiles = st_build_tiles(self.h, self.cam, self.tile, self.stream)
        return self.tiles

    def trace(self, opts=None, counters: bool = True):
        if counters:
            self.counters.zero_()
        st_trace(self.h, self.cam, self.tiles, opts, self.depth, self.normal, self.evals, self.flags,
                 self.counters if counters else None, self.stream)

    def render(self, opts=None, counters: bool = True):
        self.build_tiles()
        self.trace(opts, counters)

    def update_prims(self, ids, params):
        st_scene_update_prims(self.h, ids, params, self.stream)

    def addresses(self):
        return st_scene_addresses(self.h, self.scene.n_nodes)

    def close(self):
        if self.h:
            st_scene_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ---- batched rendering and the autotuner ---------------------------------------------
def st_tune_key(n_prims: int, width: int, height: int, step_mode: int = ST_STEP_PLAIN) -> str:
    buf = C.create_string_buffer(96)
    _check(_lib.st_tune_key(n_prims, width, height, step_mode, buf, 96), "st_tune_key")
    return buf.value.decode()


def st_tune_load(path, key: str) -> st_tune | None:
    """The cached entry, or None when the file or key is absent."""
    t = st_tune()
    rc = _lib.st_tune_load(str(path).encode(), key.encode(), C.byref(t))
    return t if rc == ST_OK else None


def st_tune_store(path, key: str, t: st_tune) -> None:
    _check(_lib.st_tune_store(str(path).encode(), key.encode(), C.byref(t)), "st_tune_store")


def st_autotune(h, cam, opts=None, cache_path=None, stream=None) -> st_tune:
    c = make_camera(cam)
    o = opts if opts is not None else make_opts()
    t = st_tune()
    _check(_lib.st_autotune(h, C.byref(c), C.byref(o), None if cache_path is None else str(cache_path).encode(),
                            C.byref(t), _stream(stream)), "st_autotune")
    return t


def _batch_arrays(handles, cams, depth, normal, evals, flags):
    n = len(handles)
    if not (len(cams) == len(depth) == len(normal) == len(evals) == len(flags) == n):
        raise ValueError("batch argument lists differ in length")
    hs = (C.c_void_p * n)(*[h.value if isinstance(h, C.c_void_p) else h for h in handles])
    cs = (st_camera * n)(*[make_camera(c) for c in cams])
    ptrs = [(C.c_void_p * n)(*[t.data_ptr() for t in lst]) for lst in (depth, normal, evals, flags)]
    return n, hs, cs, ptrs


def st_batch_create(handles, cams, opts, depth, normal, evals, flags, autotune_cache=None, stream=None):
    """Plans a batch (CUDA graph).  Output lists: one torch CUDA tensor per scene."""
    n, hs, cs, ptrs = _batch_arrays(handles, cams, depth, normal, evals, flags)
    o = opts if opts is not None else make_opts()
    b = C.c_void_p()
    _check(_lib.st_batch_create(hs, cs, n, C.byref(o), *ptrs,
                                None if autotune_cache is None else str(autotune_cache).encode(), C.byref(b),
                                _stream(stream)), "st_batch_create")
    return b


def st_batch_render(b, counters: bool = False):
    """Replays the batch graph; returns the host counters when asked."""
    if counters:
        out = np.zeros(ST_NUM_COUNTERS, np.uint64)
        _check(_lib.st_batch_render(b, out.ctypes.data), "st_batch_render")
        return out
    _check(_lib.st_batch_render(b, None), "st_batch_render")
    return None


def st_batch_tiles(b, i: int) -> int:
    return _lib.st_batch_tiles(b, i)


def st_batch_graph_kernels(b) -> int:
    return _lib.st_batch_graph_kernels(b)


def st_batch_destroy(b) -> None:
    _lib.st_batch_destroy(b)


def st_render_batch(handles, cams, opts, depth, normal, evals, flags, autotune_cache=None, stream=None) -> None:
    n, hs, cs, ptrs = _batch_arrays(handles, cams, depth, normal, evals, flags)
    o = opts if opts is not None else make_opts()
    _check(_lib.st_render_batch(hs, cs, n, C.byref(o), *ptrs,
                                None if autotune_cache is None else str(autotune_cache).encode(), _stream(stream)),
           "st_render_batch")
