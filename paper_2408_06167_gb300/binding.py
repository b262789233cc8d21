"""Thin ctypes binding of libblindmatch.so: the C-ABI of include/blindmatch.h
under the same names, marshalling numpy arrays and handles only.  Every step
of the match runs in the CUDA library; there is no Python or CPU fallback: if
the library cannot be loaded, importing this module raises.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_LIB_PATH = _build.LIB
if not os.path.exists(_LIB_PATH):
    raise ImportError(f"libblindmatch.so is not built ({_LIB_PATH}); run paper_2408_06167_gb300/build.py")
_L = ctypes.CDLL(_LIB_PATH)

_vp = ctypes.c_void_p
_u32, _u64, _i32, _i64, _dbl = ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_U64P = ctypes.POINTER(ctypes.c_uint64)
_I64P = ctypes.POINTER(ctypes.c_int64)
_I32P = ctypes.POINTER(ctypes.c_int32)
_U32P = ctypes.POINTER(ctypes.c_uint32)
_DP = ctypes.POINTER(ctypes.c_double)
_PP = ctypes.POINTER(ctypes.c_void_p)

BM_QUERY_TILED = 0
BM_QUERY_EXPANDED = 1
BM_QUERY_TEMPLATE = 2
BM_PACK_REAL = 0
BM_PACK_COMPLEX = 1
BM_LAYOUT_ENCRYPTED = 0x100
BM_LAYOUT_HOISTED = 0x200
BM_LAYOUT_HOISTED_ROTSUM = 0x400
BM_LAYOUT_HOISTED_COMPRESSION = 0x800
BM_LAYOUT_DOUBLE_HOISTED = 0x1000
BM_LAYOUT_FUSED_EXPANSION = 0x2000
BM_LAYOUT_DEFERRED_DIVISION = 0x4000
BM_LAYOUT_FUSED_COMPRESSION = 0x8000
BM_SCHED_HOISTED_EXPANSION = 1
BM_SCHED_HOISTED_ROTSUM = 2
BM_SCHED_HOISTED_COMPRESSION = 4
BM_SCHED_ALL = 7                      # every hoisted form, one ModDown per rotation
BM_SCHED_DOUBLE_HOISTED = 8
BM_SCHED_FUSED_EXPANSION = 16
BM_SCHED_DEFERRED_DIVISION = 32
BM_SCHED_FUSED_COMPRESSION = 64
BM_KEYS_ENCRYPTED_GALLERY = 1
BM_KEYS_HOISTED = 2
BM_EXPAND_DOUBLING = 0
BM_EXPAND_HOISTED = 1
BM_EXPAND_FUSED = 2
BM_EXPAND_DEFERRED = 3
BM_ENC_KEEP_DEVICE = 1
PRESETS = {"toy": 0, "ring16": 1, "small4": 2}
STATUS = ["BM_OK", "BM_E_ARG", "BM_E_PARAM", "BM_E_LEVEL", "BM_E_KEY_MISSING", "BM_E_DIM", "BM_E_OOM",
          "BM_E_HBM_BUDGET", "BM_E_CUDA", "BM_E_TIMEOUT", "BM_E_CANCELLED", "BM_E_FORMAT"]


class bm_server_stats_t(ctypes.Structure):
    _fields_ = [("submitted", _u64), ("completed", _u64), ("failed", _u64), ("cancelled", _u64),
                ("batches", _u64), ("mean_batch", _dbl), ("p50_ms", _dbl), ("p99_ms", _dbl),
                ("matches_per_s", _dbl), ("workspace_bytes", _u64)]


class bm_params(ctypes.Structure):
    _fields_ = [("log_n", _u32), ("n_q", _u32), ("q_bits", _u32 * 6), ("n_p", _u32), ("p_bits", _u32 * 3),
                ("dnum", _u32), ("log_scale", _u32), ("secret_hw", _u32), ("sigma", _dbl)]


OPS = {"rotate": 0, "rescale": 1, "mul_plain": 2, "mac": 3, "ntt": 4, "intt": 5, "copy": 6, "mac_ct": 7,
       "modup": 8, "rot_hoisted": 9, "mac_circ": 10, "accum": 11, "ip_sum": 12, "moddown": 13}
OP_NAMES = {v: k for k, v in OPS.items()}
BM_OP_KINDS = 14
BM_MAX_Q = 6
BM_COST_POINTS = 8


class bm_op_launch(ctypes.Structure):
    _fields_ = [("op", _u32), ("level", _u32), ("count", _u32), ("queries", _u32), ("parts", _u32)]


class bm_op_costs(ctypes.Structure):
    _fields_ = [("units", (_dbl * BM_COST_POINTS) * BM_OP_KINDS),
                ("t_us", ((_dbl * BM_COST_POINTS) * BM_MAX_Q) * BM_OP_KINDS)]

    def as_arrays(self):
        """(units[op][k], t_us[op][level][k]) as numpy arrays."""
        u = np.ctypeslib.as_array(self.units).copy()
        t = np.ctypeslib.as_array(self.t_us).copy()
        return u, t

    @classmethod
    def from_arrays(cls, units, t_us):
        c = cls()
        np.ctypeslib.as_array(c.units)[...] = units
        np.ctypeslib.as_array(c.t_us)[...] = t_us
        return c


_SIGS = {
    "bm_last_error": (ctypes.c_char_p, []),
    "bm_params_preset": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(bm_params)]),
    "bm_context_create": (ctypes.c_int, [ctypes.POINTER(bm_params), ctypes.c_int, _PP]),
    "bm_context_destroy": (None, [_vp]),
    "bm_context_primes": (ctypes.c_int, [_vp, _U64P, ctypes.c_size_t]),
    "bm_keygen": (ctypes.c_int, [_vp, _u64, _u32, _u32, _PP, _PP, _PP]),
    "bm_keygen_ex": (ctypes.c_int, [_vp, _u64, _u32, _u32, _u32, _PP, _PP, _PP]),
    "bm_enroll_encrypted": (ctypes.c_int, [_vp, _vp, _PP, _u64, _u32, _u32, _PP]),
    "bm_encrypt_batch": (ctypes.c_int, [_vp, _vp, _DP, _u64, _u32, _u32, _u32, _u64, _u64, _u32, _PP]),
    "bm_gallery_import_encrypted": (ctypes.c_int, [_vp, _U64P, _U64P, _U64P, _u64, _u32, _u32, _PP]),
    "bm_gallery_info": (ctypes.c_int, [_vp, _U32P, _U32P]),
    "bm_gallery_set_expansion": (ctypes.c_int, [_vp, _u32]),
    "bm_gallery_set_schedule": (ctypes.c_int, [_vp, _u32]),
    "bm_secret_key_destroy": (None, [_vp]),
    "bm_public_key_destroy": (None, [_vp]),
    "bm_eval_keys_destroy": (None, [_vp]),
    "bm_eval_keys_rotations": (ctypes.c_int, [_vp, _I32P, ctypes.c_size_t, _U32P]),
    "bm_secret_key_export": (ctypes.c_int, [_vp, _I64P, ctypes.c_size_t]),
    "bm_public_key_export": (ctypes.c_int, [_vp, _U64P, ctypes.c_size_t]),
    "bm_eval_keys_export": (ctypes.c_int, [_vp, _i32, _U64P, ctypes.c_size_t]),
    "bm_encode_gallery": (ctypes.c_int, [_vp, _DP, _u64, _u32, _u32, _PP]),
    "bm_gallery_import": (ctypes.c_int, [_vp, _U64P, _U64P, _U64P, _u64, _u32, _u32, _PP]),
    "bm_gallery_layout": (ctypes.c_int, [_vp, _u64, _u32, _u32, _U32P, _U32P, _U32P, _U32P, _U32P]),
    "bm_gallery_layout_packed": (ctypes.c_int, [_vp, _u64, _u32, _u32, _u32, _U32P, _U32P, _U32P, _U32P, _U32P]),
    "bm_encode_gallery_packed": (ctypes.c_int, [_vp, _DP, _u64, _u32, _u32, _u32, _PP]),
    "bm_gallery_import_packed": (ctypes.c_int, [_vp, _U64P, _U64P, _U64P, _u64, _u32, _u32, _u32, _PP]),
    "bm_gallery_export": (ctypes.c_int, [_vp, _U64P, _U64P, _U64P]),
    "bm_gallery_destroy": (None, [_vp]),
    "bm_encrypt_query": (ctypes.c_int, [_vp, _vp, _DP, _u32, _u32, _u32, _u64, _u64, _PP]),
    "bm_ciphertext_import": (ctypes.c_int, [_vp, _U64P, _u32, _u32, _PP]),
    "bm_ciphertext_info": (ctypes.c_int, [_vp, _U32P, _U32P]),
    "bm_ciphertext_export": (ctypes.c_int, [_vp, _U64P, ctypes.c_size_t]),
    "bm_ciphertext_upload": (ctypes.c_int, [_vp, _vp]),
    "bm_ciphertext_destroy": (None, [_vp]),
    "bm_match": (ctypes.c_int, [_vp, _vp, _vp, _PP, _u32, _vp, _PP]),
    "bm_match_async": (ctypes.c_int, [_vp, _vp, _vp, _PP, _u32, _vp, _PP]),
    "bm_result_info": (ctypes.c_int, [_vp, _U32P, _U32P, _U32P]),
    "bm_result_export": (ctypes.c_int, [_vp, _u32, _U64P, ctypes.c_size_t]),
    "bm_result_destroy": (None, [_vp]),
    "bm_decrypt_scores": (ctypes.c_int, [_vp, _vp, _vp, _u32, _DP, _u64, _I64P, _DP]),
    "bm_poly_mul": (ctypes.c_int, [_vp, _U64P, _U64P, _U64P, _u32]),
    "bm_ct_rotate": (ctypes.c_int, [_vp, _vp, _vp, _i32, _PP]),
    "bm_ct_rescale": (ctypes.c_int, [_vp, _vp, _PP]),
    "bm_ntt_forward": (ctypes.c_int, [_vp, _vp, _u32, _u32, _vp]),
    "bm_ntt_inverse": (ctypes.c_int, [_vp, _vp, _u32, _u32, _vp]),
    "bm_ct_rotate_noalloc": (ctypes.c_int, [_vp, _vp, _vp, _u32, _u32, _i32, _vp, _vp]),
    "bm_server_create": (ctypes.c_int, [_vp, _u64, _u32, _u32, _PP]),
    "bm_server_destroy": (None, [_vp]),
    "bm_server_add_gallery": (ctypes.c_int, [_vp, _vp, _vp, _U32P]),
    "bm_server_submit": (ctypes.c_int, [_vp, _u32, _vp, ctypes.POINTER(ctypes.c_uint64)]),
    "bm_server_wait": (ctypes.c_int, [_vp, _u64, _u32, _PP]),
    "bm_server_cancel": (ctypes.c_int, [_vp, _u64]),
    "bm_server_stats": (ctypes.c_int, [_vp, ctypes.POINTER(bm_server_stats_t)]),
    "bm_server_reset_stats": (ctypes.c_int, [_vp]),
    "bm_plan_estimate": (ctypes.c_int, [ctypes.POINTER(bm_params), _u64, _u32, _u32, _u32, _u32,
                                        ctypes.POINTER(bm_op_launch), ctypes.c_size_t,
                                        ctypes.POINTER(ctypes.c_size_t), _U64P]),
    "bm_predict_match": (ctypes.c_int, [ctypes.POINTER(bm_params), ctypes.POINTER(bm_op_costs), _u64, _u32, _u32,
                                        _u32, _u32, _DP, _U64P]),
    "bm_choose_part": (ctypes.c_int, [ctypes.POINTER(bm_params), ctypes.POINTER(bm_op_costs), _u64, _u32, _u32,
                                      _u32, _u64, _U32P, _DP]),
    "bm_measure_op_costs": (ctypes.c_int, [_vp, ctypes.POINTER(bm_op_costs)]),
    "bm_autotune_keyswitch": (ctypes.c_int, [_vp, _U32P, ctypes.c_size_t]),
    "bm_set_ks_wide_batch": (ctypes.c_int, [_vp, _u32, _u32]),
    "bm_autotune_ntt": (ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_uint8), ctypes.c_size_t]),
    "bm_set_ntt_shape": (ctypes.c_int, [_vp, _u32, _u32]),
    "bm_choose_dnum": (ctypes.c_int, [ctypes.POINTER(bm_params), ctypes.c_int, _u64, _u32, _u32, _u32, _u32, _U32P,
                                      _DP, ctypes.c_size_t]),
    "bm_profile_control": (ctypes.c_int, [_u32, _u32]),
    "bm_profile_read": (ctypes.c_int, [_u32, _U64P, _DP, _DP, _DP]),
}
for _name, (_res, _args) in _SIGS.items():
    _fn = getattr(_L, _name)
    _fn.restype = _res
    _fn.argtypes = _args


class BlindMatchError(RuntimeError):
    def __init__(self, status, msg):
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{name}: {msg}")
        self.status = status


def _check(st):
    if st != 0:
        raise BlindMatchError(st, _L.bm_last_error().decode())


def _u64p(a):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(_U64P)


class _Handle:
    """Owns one opaque handle; frees it with its _destroy call."""
    _destroy = None

    def __init__(self, ptr, owner=None):
        self.ptr = ptr
        self.owner = owner      # keeps the context alive

    def __del__(self):
        if self.ptr and self._destroy:
            getattr(_L, self._destroy)(self.ptr)
            self.ptr = None


class Context(_Handle):
    _destroy = "bm_context_destroy"


class SecretKey(_Handle):
    _destroy = "bm_secret_key_destroy"


class PublicKey(_Handle):
    _destroy = "bm_public_key_destroy"


class EvalKeys(_Handle):
    _destroy = "bm_eval_keys_destroy"


class Gallery(_Handle):
    _destroy = "bm_gallery_destroy"


class Ciphertext(_Handle):
    _destroy = "bm_ciphertext_destroy"


class Result(_Handle):
    _destroy = "bm_result_destroy"


class Server(_Handle):
    _destroy = "bm_server_destroy"


def _out():
    return ctypes.c_void_p()


# ---- the C-ABI under its own names ----

def bm_params_preset(name):
    p = bm_params()
    _check(_L.bm_params_preset(PRESETS[name] if isinstance(name, str) else name, ctypes.byref(p)))
    return p


def bm_context_create(params, device=0):
    if isinstance(params, (str, int)):
        params = bm_params_preset(params)
    h = _out()
    _check(_L.bm_context_create(ctypes.byref(params), device, ctypes.byref(h)))
    ctx = Context(h.value)
    ctx.params = params
    ctx.n = 1 << params.log_n
    ctx.n_q, ctx.n_p, ctx.dnum = params.n_q, params.n_p, params.dnum
    return ctx


def bm_context_primes(ctx):
    out = np.zeros(ctx.n_q + ctx.n_p, dtype=np.uint64)
    _check(_L.bm_context_primes(ctx.ptr, _u64p(out), out.size))
    return [int(x) for x in out]


def bm_keygen(ctx, seed, dim, part):
    return bm_keygen_ex(ctx, seed, dim, part, 0)


def bm_keygen_ex(ctx, seed, dim, part, flags):
    sk, pk, ek = _out(), _out(), _out()
    _check(_L.bm_keygen_ex(ctx.ptr, seed, dim, part, flags, ctypes.byref(sk), ctypes.byref(pk), ctypes.byref(ek)))
    return SecretKey(sk.value, ctx), PublicKey(pk.value, ctx), EvalKeys(ek.value, ctx)


def bm_eval_keys_rotations(evk):
    cnt = _u32()
    _check(_L.bm_eval_keys_rotations(evk.ptr, None, 0, ctypes.byref(cnt)))
    out = (ctypes.c_int32 * max(cnt.value, 1))()
    _check(_L.bm_eval_keys_rotations(evk.ptr, out, cnt.value, ctypes.byref(cnt)))
    return sorted(out[i] for i in range(cnt.value))


def bm_secret_key_export(sk):
    ctx = sk.owner
    out = np.zeros(ctx.n, dtype=np.int64)
    _check(_L.bm_secret_key_export(sk.ptr, out.ctypes.data_as(_I64P), out.size))
    return out


def bm_public_key_export(pk):
    ctx = pk.owner
    out = np.zeros((2, ctx.n_q, ctx.n), dtype=np.uint64)
    _check(_L.bm_public_key_export(pk.ptr, _u64p(out), out.size))
    return out


def bm_eval_keys_export(evk, rotation):
    ctx = evk.owner
    out = np.zeros((ctx.dnum, 2, ctx.n_q + ctx.n_p, ctx.n), dtype=np.uint64)
    _check(_L.bm_eval_keys_export(evk.ptr, rotation, _u64p(out), out.size))
    return out


def bm_gallery_layout(ctx, n_ids, dim, part):
    v = [_u32() for _ in range(5)]
    _check(_L.bm_gallery_layout(ctx.ptr, n_ids, dim, part, *[ctypes.byref(x) for x in v]))
    return dict(zip(["groups", "level", "tiled", "compressed", "n_out"], [x.value for x in v]))


def bm_gallery_layout_packed(ctx, n_ids, dim, part, packing):
    v = [_u32() for _ in range(5)]
    _check(_L.bm_gallery_layout_packed(ctx.ptr, n_ids, dim, part, packing, *[ctypes.byref(x) for x in v]))
    return dict(zip(["groups", "level", "tiled", "compressed", "n_out"], [x.value for x in v]))


def bm_encode_gallery(ctx, feats, dim, part):
    return bm_encode_gallery_packed(ctx, feats, dim, part, BM_PACK_REAL)


def bm_encode_gallery_packed(ctx, feats, dim, part, packing):
    f = np.ascontiguousarray(feats, dtype=np.float64)
    h = _out()
    _check(_L.bm_encode_gallery_packed(ctx.ptr, f.ctypes.data_as(_DP), f.shape[0], dim, part, packing,
                                       ctypes.byref(h)))
    g = Gallery(h.value, ctx)
    g.n_ids, g.dim, g.part, g.packing = f.shape[0], dim, part, packing
    return g


def bm_gallery_import(ctx, pts, masks, cmask, n_ids, dim, part):
    return bm_gallery_import_packed(ctx, pts, masks, cmask, n_ids, dim, part, BM_PACK_REAL)


def bm_gallery_import_packed(ctx, pts, masks, cmask, n_ids, dim, part, packing):
    arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.uint64) for a in (pts, masks, cmask)]
    ptrs = [None if a is None else _u64p(a) for a in arrs]
    h = _out()
    _check(_L.bm_gallery_import_packed(ctx.ptr, *ptrs, n_ids, dim, part, packing, ctypes.byref(h)))
    g = Gallery(h.value, ctx)
    g.n_ids, g.dim, g.part, g.packing = n_ids, dim, part, packing
    return g


def bm_encrypt_batch(ctx, pk, vectors, dim, part, mode, seed, first_id=0, flags=0):
    """Ciphertext handles of every row of `vectors` (as bm_encrypt_query with query ids first_id + k)."""
    v = np.ascontiguousarray(vectors, dtype=np.float64)
    n = v.shape[0]
    arr = (ctypes.c_void_p * n)()
    _check(_L.bm_encrypt_batch(ctx.ptr, pk.ptr, v.ctypes.data_as(_DP), n, dim, part, mode, seed, first_id, flags,
                               arr))
    return [Ciphertext(arr[k], ctx) for k in range(n)]


def bm_enroll_encrypted(ctx, evk, templates, dim, part):
    arr = (ctypes.c_void_p * len(templates))(*[t.ptr for t in templates])
    h = _out()
    _check(_L.bm_enroll_encrypted(ctx.ptr, evk.ptr, arr, len(templates), dim, part, ctypes.byref(h)))
    g = Gallery(h.value, ctx)
    g.n_ids, g.dim, g.part, g.packing, g.encrypted = len(templates), dim, part, BM_PACK_REAL, True
    return g


def bm_gallery_import_encrypted(ctx, cts, masks, cmask, n_ids, dim, part):
    arrs = [np.ascontiguousarray(a, dtype=np.uint64) for a in (cts, masks, cmask)]
    h = _out()
    _check(_L.bm_gallery_import_encrypted(ctx.ptr, *[_u64p(a) for a in arrs], n_ids, dim, part, ctypes.byref(h)))
    g = Gallery(h.value, ctx)
    g.n_ids, g.dim, g.part, g.packing, g.encrypted = n_ids, dim, part, BM_PACK_REAL, True
    return g


def bm_gallery_set_expansion(g, mode):
    _check(_L.bm_gallery_set_expansion(g.ptr, mode))
    g.hoisted = mode in (BM_EXPAND_HOISTED, BM_EXPAND_FUSED, BM_EXPAND_DEFERRED)


def bm_gallery_set_schedule(g, flags):
    _check(_L.bm_gallery_set_schedule(g.ptr, flags))
    g.hoisted = bool(flags & BM_SCHED_HOISTED_EXPANSION)


def bm_gallery_info(g):
    """(encrypted, packing)."""
    e, p = _u32(), _u32()
    _check(_L.bm_gallery_info(g.ptr, ctypes.byref(e), ctypes.byref(p)))
    return bool(e.value), p.value


def bm_gallery_export(g):
    ctx = g.owner
    enc = getattr(g, "encrypted", False)
    lo = bm_gallery_layout_packed(ctx, g.n_ids, g.dim, g.part, g.packing | (BM_LAYOUT_ENCRYPTED if enc else 0))
    n_in, lvl = g.dim // g.part, lo["level"]
    shape = (lo["groups"], n_in, 2, lvl + 1, ctx.n) if enc else (lo["groups"], n_in, lvl + 1, ctx.n)
    pts = np.zeros(shape, dtype=np.uint64)
    masks = np.zeros((n_in, ctx.n_q, ctx.n), dtype=np.uint64) if lo["tiled"] else None
    cmask = np.zeros((lvl, ctx.n), dtype=np.uint64) if lo["compressed"] else None
    _check(_L.bm_gallery_export(g.ptr, _u64p(pts), None if masks is None else _u64p(masks),
                                None if cmask is None else _u64p(cmask)))
    return pts, masks, cmask


def bm_encrypt_query(ctx, pk, q, dim, part, mode, seed, query_id):
    qa = np.ascontiguousarray(q, dtype=np.float64)
    h = _out()
    _check(_L.bm_encrypt_query(ctx.ptr, pk.ptr, qa.ctypes.data_as(_DP), dim, part, mode, seed, query_id,
                               ctypes.byref(h)))
    return Ciphertext(h.value, ctx)


def bm_ciphertext_import(ctx, data, level):
    d = np.ascontiguousarray(data, dtype=np.uint64).reshape(-1, 2, level + 1, ctx.n)
    h = _out()
    _check(_L.bm_ciphertext_import(ctx.ptr, _u64p(d), d.shape[0], level, ctypes.byref(h)))
    return Ciphertext(h.value, ctx)


def bm_ciphertext_info(ct):
    n, l = _u32(), _u32()
    _check(_L.bm_ciphertext_info(ct.ptr, ctypes.byref(n), ctypes.byref(l)))
    return n.value, l.value


def bm_ciphertext_export(ct):
    n_cts, level = bm_ciphertext_info(ct)
    out = np.zeros((n_cts, 2, level + 1, ct.owner.n), dtype=np.uint64)
    _check(_L.bm_ciphertext_export(ct.ptr, _u64p(out), out.size))
    return out


def bm_ciphertext_upload(ct, stream=None):
    _check(_L.bm_ciphertext_upload(ct.ptr, stream))


def bm_match(ctx, evk, gallery, queries, stream=None):
    arr = (ctypes.c_void_p * len(queries))(*[q.ptr for q in queries])
    h = _out()
    _check(_L.bm_match(ctx.ptr, evk.ptr, gallery.ptr, arr, len(queries), stream, ctypes.byref(h)))
    return Result(h.value, ctx)


def bm_match_async(ctx, evk, gallery, queries, stream=None):
    """bm_match without the wait: the result is complete once `stream` has passed the
    call (export and decryption wait for it themselves)."""
    arr = (ctypes.c_void_p * len(queries))(*[q.ptr for q in queries])
    h = _out()
    _check(_L.bm_match_async(ctx.ptr, evk.ptr, gallery.ptr, arr, len(queries), stream, ctypes.byref(h)))
    return Result(h.value, ctx)


def bm_result_info(r):
    a, b, c = _u32(), _u32(), _u32()
    _check(_L.bm_result_info(r.ptr, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, bool(c.value)


def bm_result_export(r, query_index, out=None):
    """Score ciphertexts of one query, [n_out][2][1][N] uint64; into `out` when given
    (a C-contiguous uint64 array of that size, e.g. a view of page-locked memory)."""
    _, n_out, _ = bm_result_info(r)
    shape = (n_out, 2, 1, r.owner.n)
    if out is None:
        out = np.empty(shape, dtype=np.uint64)
    elif out.dtype != np.uint64 or not out.flags.c_contiguous or out.size != int(np.prod(shape)):
        raise ValueError(f"out must be a C-contiguous uint64 array of {shape}")
    _check(_L.bm_result_export(r.ptr, query_index, _u64p(out), out.size))
    return out.reshape(shape)


def bm_decrypt_scores(ctx, sk, r, query_index, n_ids):
    scores = np.zeros(n_ids, dtype=np.float64)
    rank1, best = _i64(), _dbl()
    _check(_L.bm_decrypt_scores(ctx.ptr, sk.ptr, r.ptr, query_index, scores.ctypes.data_as(_DP), n_ids,
                                ctypes.byref(rank1), ctypes.byref(best)))
    return scores, rank1.value, best.value


def bm_poly_mul(ctx, a, b):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    out = np.zeros_like(a)
    _check(_L.bm_poly_mul(ctx.ptr, _u64p(a), _u64p(b), _u64p(out), a.shape[0]))
    return out


def bm_ct_rotate(ctx, evk, ct, rotation):
    h = _out()
    _check(_L.bm_ct_rotate(ctx.ptr, evk.ptr, ct.ptr, rotation, ctypes.byref(h)))
    return Ciphertext(h.value, ctx)


def bm_ct_rescale(ctx, ct):
    h = _out()
    _check(_L.bm_ct_rescale(ctx.ptr, ct.ptr, ctypes.byref(h)))
    return Ciphertext(h.value, ctx)


def bm_ct_rotate_noalloc(ctx, evk, d_in, n_cts, level, rotation, d_out, stream=None):
    """Rotation on caller-provided device buffers (integer device pointers), no device allocation."""
    _check(_L.bm_ct_rotate_noalloc(ctx.ptr, evk.ptr, d_in, n_cts, level, rotation, d_out, stream))


def bm_ntt_forward(ctx, d_ptr, n_polys, n_limbs, stream=None):
    _check(_L.bm_ntt_forward(ctx.ptr, d_ptr, n_polys, n_limbs, stream))


def bm_ntt_inverse(ctx, d_ptr, n_polys, n_limbs, stream=None):
    _check(_L.bm_ntt_inverse(ctx.ptr, d_ptr, n_polys, n_limbs, stream))


KERNEL_KINDS = ["ntt", "modup", "ks_ip", "moddown", "ks_combine", "rescale", "mac", "mul_plain", "other"]


def bm_profile_control(timing, reset):
    _check(_L.bm_profile_control(int(timing), int(reset)))


def bm_profile_read(kind):
    """(launches, device_ms, algorithmic_bytes, algorithmic_32bit_mul_ops) of one kernel class."""
    k = KERNEL_KINDS.index(kind) if isinstance(kind, str) else kind
    n, ms, by, ops = _u64(), _dbl(), _dbl(), _dbl()
    _check(_L.bm_profile_read(k, ctypes.byref(n), ctypes.byref(ms), ctypes.byref(by), ctypes.byref(ops)))
    return n.value, ms.value, by.value, ops.value


def bm_server_create(ctx, hbm_budget_bytes, max_batch=64, executors=2):
    h = _out()
    _check(_L.bm_server_create(ctx.ptr, hbm_budget_bytes, max_batch, executors, ctypes.byref(h)))
    return Server(h.value, ctx)


def bm_server_add_gallery(srv, gallery, evk):
    gid = _u32()
    _check(_L.bm_server_add_gallery(srv.ptr, gallery.ptr, evk.ptr, ctypes.byref(gid)))
    srv.keep = getattr(srv, "keep", []) + [gallery, evk]      # borrowed by the server: keep alive
    return gid.value


def bm_server_submit(srv, gid, query):
    t = ctypes.c_uint64()
    _check(_L.bm_server_submit(srv.ptr, gid, query.ptr, ctypes.byref(t)))
    return t.value


def bm_server_wait(srv, ticket, timeout_ms=60000):
    h = _out()
    _check(_L.bm_server_wait(srv.ptr, ticket, timeout_ms, ctypes.byref(h)))
    return Result(h.value, srv.owner)


def bm_server_cancel(srv, ticket):
    _check(_L.bm_server_cancel(srv.ptr, ticket))


def bm_server_stats(srv):
    st = bm_server_stats_t()
    _check(_L.bm_server_stats(srv.ptr, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in bm_server_stats_t._fields_}


def bm_server_reset_stats(srv):
    _check(_L.bm_server_reset_stats(srv.ptr))


# ---- schedule model, part-size choice, kernel-shape tuning ----

def _params(p):
    return bm_params_preset(p) if isinstance(p, (str, int)) else p


def bm_plan_estimate(params, n_ids, dim, part, n_queries, packing=BM_PACK_REAL):
    """(launches as a list of dicts, plan bytes) of the match; host only."""
    p = _params(params)
    n = ctypes.c_size_t()
    _check(_L.bm_plan_estimate(ctypes.byref(p), n_ids, dim, part, packing, n_queries, None, 0, ctypes.byref(n),
                               None))
    arr = (bm_op_launch * max(n.value, 1))()
    nbytes = _u64()
    _check(_L.bm_plan_estimate(ctypes.byref(p), n_ids, dim, part, packing, n_queries, arr, n.value,
                               ctypes.byref(n), ctypes.byref(nbytes)))
    ops = [dict(op=OP_NAMES[a.op], level=a.level, count=a.count, queries=a.queries, parts=a.parts)
           for a in arr[:n.value]]
    return ops, nbytes.value


def bm_predict_match(params, costs, n_ids, dim, part, n_queries, packing=BM_PACK_REAL):
    """(predicted ms, plan bytes); host only."""
    p = _params(params)
    ms, nbytes = _dbl(), _u64()
    _check(_L.bm_predict_match(ctypes.byref(p), ctypes.byref(costs), n_ids, dim, part, packing, n_queries,
                               ctypes.byref(ms), ctypes.byref(nbytes)))
    return ms.value, nbytes.value


def bm_choose_part(params, costs, n_ids, dim, n_queries, hbm_budget=0, packing=BM_PACK_REAL):
    """(part size, predicted ms); host only."""
    p = _params(params)
    part, ms = _u32(), _dbl()
    _check(_L.bm_choose_part(ctypes.byref(p), ctypes.byref(costs), n_ids, dim, packing, n_queries, hbm_budget,
                             ctypes.byref(part), ctypes.byref(ms)))
    return part.value, ms.value


def bm_measure_op_costs(ctx):
    c = bm_op_costs()
    _check(_L.bm_measure_op_costs(ctx.ptr, ctypes.byref(c)))
    return c


def bm_autotune_keyswitch(ctx):
    """Per-level batch size from which rotations use 16 coefficients per thread (2^30 = never)."""
    out = (_u32 * ctx.n_q)()
    _check(_L.bm_autotune_keyswitch(ctx.ptr, out, ctx.n_q))
    return list(out)


def bm_set_ks_wide_batch(ctx, level, batch):
    _check(_L.bm_set_ks_wide_batch(ctx.ptr, level, batch))


BM_NTT_BUCKETS = 10


def bm_autotune_ntt(ctx):
    """Per batch bucket (limbs <= 2^k) the standalone NTT shape the tuner keeps (0, 1, 2)."""
    out = (ctypes.c_uint8 * BM_NTT_BUCKETS)()
    _check(_L.bm_autotune_ntt(ctx.ptr, out, BM_NTT_BUCKETS))
    return list(out)


def bm_set_ntt_shape(ctx, bucket, shape):
    _check(_L.bm_set_ntt_shape(ctx.ptr, bucket, shape))


def bm_choose_dnum(params, n_ids, dim, part, n_queries, packing=BM_PACK_REAL, device=0):
    """(dnum of least predicted match time, predicted ms per dnum 1..4 (0: not taken))."""
    p = _params(params)
    d = _u32()
    ms = (ctypes.c_double * 4)()
    _check(_L.bm_choose_dnum(ctypes.byref(p), device, n_ids, dim, part, packing, n_queries, ctypes.byref(d), ms, 4))
    return d.value, list(ms)
