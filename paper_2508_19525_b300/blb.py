"""ctypes binding of libblb.so (include/blb.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  Device memory comes from PyTorch's caching allocator, installed with
blb_set_allocator; streams are PyTorch streams.  There is no CPU fallback: if
the library is missing or no GPU is present, the calls raise.
"""
import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libblb.so")

OK, ERR_ARG, ERR_LEVEL, ERR_SCALE, ERR_NO_KEY, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_PARAM = 0, -1, -2, -3, -4, -5, -6, -7, -8

_vp = ctypes.c_void_p
_u32 = ctypes.c_uint32
_u64 = ctypes.c_uint64
_i32 = ctypes.c_int32
_dbl = ctypes.c_double
_pp = ctypes.POINTER(ctypes.c_void_p)


class BlbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"blb error {code}: {msg}")
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [("logN", _u32), ("nQ", _u32), ("nP", _u32), ("q_bits", ctypes.POINTER(_u32)),
                ("p_bits", ctypes.POINTER(_u32)), ("dnum", _u32), ("scale", _dbl)]


class _Sched(ctypes.Structure):
    _fields_ = [("b1", _u32)]


class _CcSched(ctypes.Structure):
    _fields_ = [("b1s1", _u32), ("b1s2", _u32), ("c_chunk", _u32), ("t_chunk", _u32), ("workspace_bytes", _u64)]


ALLOC_FN = ctypes.CFUNCTYPE(_vp, ctypes.c_size_t, _vp, _vp)
FREE_FN = ctypes.CFUNCTYPE(None, _vp, ctypes.c_size_t, _vp, _vp)

# every function of include/blb.h with its ctypes signature
SIGNATURES = {
    "blb_set_allocator": (ctypes.c_int, [ALLOC_FN, FREE_FN, _vp]),
    "blb_last_error": (ctypes.c_char_p, []),
    "blb_version": (ctypes.c_char_p, []),
    "blb_params_primes": (ctypes.c_int, [ctypes.POINTER(_Params), _vp]),
    "blb_ctx_create": (ctypes.c_int, [ctypes.POINTER(_Params), _vp, _pp]),
    "blb_ctx_free": (None, [_vp]),
    "blb_ctx_info": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "blb_ctx_primes": (ctypes.c_int, [_vp, _vp]),
    "blb_ctx_sync": (ctypes.c_int, [_vp]),
    "blb_ctx_bytes_in_use": (_u64, [_vp]),
    "blb_keygen": (ctypes.c_int, [_vp, _u64, _vp, _u32, ctypes.c_int, _pp]),
    "blb_keys_free": (None, [_vp]),
    "blb_keys_export": (ctypes.c_int, [_vp, _vp, ctypes.c_int, _i32, _vp]),
    "blb_encode": (ctypes.c_int, [_vp, _vp, _u64, _u32, _dbl, _pp]),
    "blb_pt_free": (None, [_vp]),
    "blb_pt_export": (ctypes.c_int, [_vp, _vp, _vp]),
    "blb_encrypt": (ctypes.c_int, [_vp, _vp, _vp, _u64, _pp]),
    "blb_ct_free": (None, [_vp]),
    "blb_ct_info": (ctypes.c_int, [_vp, _vp, _vp, _vp]),
    "blb_ct_export": (ctypes.c_int, [_vp, _vp, _vp]),
    "blb_ct_import": (ctypes.c_int, [_vp, _vp, _u32, _u32, _dbl, _pp]),
    "blb_decrypt": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp]),
    "blb_ct_copy": (ctypes.c_int, [_vp, _vp, _vp]),
    "blb_encode_batch": (ctypes.c_int, [_vp, _vp, _u64, _u32, _u32, _dbl, _vp]),
    "blb_encrypt_batch": (ctypes.c_int, [_vp, _vp, _vp, _u32, _vp, _vp]),
    "blb_he2mpc_batch": (ctypes.c_int, [_vp, _vp, _vp, _u32, _vp, _vp, _vp]),
    "blb_decrypt_batch": (ctypes.c_int, [_vp, _vp, _vp, _u32, _vp, _vp]),
    "blb_rotate": (ctypes.c_int, [_vp, _vp, _vp, _i32, _pp]),
    "blb_rescale": (ctypes.c_int, [_vp, _vp]),
    "blb_add": (ctypes.c_int, [_vp, _vp, _vp, _pp]),
    "blb_mul_plain": (ctypes.c_int, [_vp, _vp, _vp, _pp]),
    "blb_sub": (ctypes.c_int, [_vp, _vp, _vp, _pp]),
    "blb_drop_level": (ctypes.c_int, [_vp, _vp, _u32, _pp]),
    "blb_mul_const": (ctypes.c_int, [_vp, _vp, _vp, _u64, _dbl, _pp]),
    "blb_mul": (ctypes.c_int, [_vp, _vp, _vp, _vp, ctypes.c_int, _pp]),
    "blb_relinearize": (ctypes.c_int, [_vp, _vp, _vp, _pp]),
    "blb_keyswitch_coeffs": (ctypes.c_int, [_vp, _vp, _i32, _vp, _u32, _vp]),
    "blb_keyswitch_noalloc": (ctypes.c_int, [_vp, _vp, _i32, _vp, _u32, _vp]),
    "blb_ctx_set_wait_limit": (ctypes.c_int, [_vp, _u64]),
    "blb_ctx_test_withhold_copies": (ctypes.c_int, [_vp, ctypes.c_int]),
    "blb_ctx_set_batch_mac": (ctypes.c_int, [_vp, ctypes.c_int]),
    "blb_cp_plan_create": (ctypes.c_int, [_vp, _u32, _u32, _vp, _u32, _u32, ctypes.POINTER(_Sched), _pp]),
    "blb_cp_plan_create_diag": (ctypes.c_int, [_vp, _u32, _u32, _vp, _u32, _vp, _u32, _u32, ctypes.POINTER(_Sched), _pp]),
    "blb_cp_plan_free": (None, [_vp]),
    "blb_cp_plan_info": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "blb_matmul_cp_plan": (ctypes.c_int, [_vp, _vp, _vp, _pp, _u32, _pp]),
    "blb_matmul_cp_batch": (ctypes.c_int, [_vp, _vp, _vp, _pp, _u32, _pp]),
    "blb_matmul_cp_multi": (ctypes.c_int, [_vp, _pp, _vp, _pp, _u32, _pp]),
    "blb_matmul_cp": (ctypes.c_int, [_vp, _vp, _pp, _u32, _u32, _u32, _vp, _u32, ctypes.POINTER(_Sched), _pp]),
    "blb_cc_plan_create": (ctypes.c_int, [_vp, _u32, _u32, _u32, _u32, ctypes.POINTER(_CcSched), _pp]),
    "blb_cc_plan_free": (None, [_vp]),
    "blb_cc_plan_info": (ctypes.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "blb_cc_plan_rotations": (ctypes.c_int, [_vp, _vp, _u32, _vp]),
    "blb_matmul_cc_plan": (ctypes.c_int, [_vp, _vp, _vp, _pp, _pp, _u32, _pp]),
    "blb_matmul_cc": (ctypes.c_int, [_vp, _vp, _pp, _pp, _u32, _u32, _u32, _u32, ctypes.POINTER(_CcSched), _pp]),
    "blb_he2mpc": (ctypes.c_int, [_vp, _vp, _vp, _u64, _pp, _vp]),
    "blb_rotate_sum_packing": (ctypes.c_int, [_vp, _vp, _pp, _u32, _u32, _u32, ctypes.c_int, ctypes.c_int, _pp]),
    "blb_layernorm_head": (ctypes.c_int, [_vp, _vp, _pp, _u32, _u32, _u32, _u32, _pp, _pp]),
    "blb_f2r_wrap_sim": (ctypes.c_int, [_vp, _vp, _vp, _u32, _u64, _vp, _vp, _vp]),
    "blb_c2m_local": (ctypes.c_int, [_vp, _u32, _vp, _vp, _u32, _dbl, _u32, _u32, _vp]),
    "blb_ext_wrap_sim": (ctypes.c_int, [_vp, _vp, _vp, _u32, _u32, _u32, _u64, _vp, _vp, _vp]),
    "blb_m2c_local": (ctypes.c_int, [_vp, _u32, _vp, _vp, _u32, _u32, _u32, _dbl, _u32, _u32, _vp]),
    "blb_pt_import": (ctypes.c_int, [_vp, _vp, _u32, _dbl, _pp]),
    "blb_add_plain": (ctypes.c_int, [_vp, _vp, _vp, _pp]),
    "blb_ntt": (ctypes.c_int, [_vp, _vp, _u32, _vp, ctypes.c_int]),
    "blb_ntt_autotune": (ctypes.c_int, [_vp, _u32, _vp, _vp, _vp]),
    "blb_ntt_set_split": (ctypes.c_int, [_vp, ctypes.c_int]),
    "blb_ntt_set_radix": (ctypes.c_int, [_vp, ctypes.c_int]),
    "blb_kernel_launches": (_u64, []),
    "blb_profile_enable": (ctypes.c_int, [_vp, ctypes.c_int]),
    "blb_profile_read": (ctypes.c_int, [_vp, ctypes.c_char_p, _vp, _vp, _vp]),
    "blb_profile_read_ops": (ctypes.c_int, [_vp, ctypes.c_char_p, _vp, _vp, _vp]),
    "blb_ctx_set_deferred_encode_check": (ctypes.c_int, [_vp, ctypes.c_int]),
    "blb_profile_select": (ctypes.c_int, [_vp, ctypes.c_char_p]),
}

_lib = None
_alloc_refs = None


def lib():
    """Load libblb.so (raises if it was not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} missing: run paper_2508_19525_b300/build.py (no CPU fallback exists)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        raise BlbError(rc, lib().blb_last_error().decode())


def kernel_launches():
    return int(lib().blb_kernel_launches())


def last_error():
    return lib().blb_last_error().decode()


def use_torch_allocator():
    """Route the library's device allocations through PyTorch's caching allocator."""
    global _alloc_refs
    import torch

    def _alloc(nbytes, stream, user):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), stream=int(stream or 0))
        except Exception:
            return None

    def _free(ptr, nbytes, stream, user):
        torch.cuda.caching_allocator_delete(ptr)

    a, f = ALLOC_FN(_alloc), FREE_FN(_free)
    _check(lib().blb_set_allocator(a, f, None))
    _alloc_refs = (a, f)


def _ptr(a):
    """Data pointer of a numpy array or torch tensor (host or device)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _params(logN, q_bits, p_bits, dnum, scale):
    qb = (_u32 * len(q_bits))(*q_bits)
    pb = (_u32 * len(p_bits))(*p_bits)
    p = _Params(logN, len(q_bits), len(p_bits), qb, pb, dnum, scale)
    return p, (qb, pb)


def params_primes(logN, q_bits, p_bits, dnum):
    """Host-only prime selection of the library (no GPU needed)."""
    p, keep = _params(logN, q_bits, p_bits, dnum, 2.0 ** 40)
    out = np.zeros(len(q_bits) + len(p_bits), np.uint64)
    _check(lib().blb_params_primes(ctypes.byref(p), out.ctypes.data))
    return [int(x) for x in out]


class _Handle:
    _free = None

    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h

    def free(self):
        if self.h:
            getattr(lib(), self._free)(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


class Keys(_Handle):
    _free = "blb_keys_free"


class Plaintext(_Handle):
    _free = "blb_pt_free"


class Ciphertext(_Handle):
    _free = "blb_ct_free"

    def info(self):
        lv, npl, sc = _u32(), _u32(), _dbl()
        _check(lib().blb_ct_info(self.h, ctypes.byref(lv), ctypes.byref(npl), ctypes.byref(sc)))
        return lv.value, npl.value, sc.value

    @property
    def level(self):
        return self.info()[0]

    @property
    def scale(self):
        return self.info()[2]


class CpPlan(_Handle):
    _free = "blb_cp_plan_free"

    def info(self):
        v = [_u32() for _ in range(4)] + [_u64()]
        _check(lib().blb_cp_plan_info(self.h, *[ctypes.byref(x) for x in v]))
        return dict(nX=v[0].value, nY=v[1].value, b1=v[2].value, G=v[3].value, plaintext_bytes=v[4].value)


class CcPlan(_Handle):
    _free = "blb_cc_plan_free"

    def info(self):
        v = [_u32() for _ in range(5)] + [_u64()] + [_u32() for _ in range(2)]
        _check(lib().blb_cc_plan_info(self.h, *[ctypes.byref(x) for x in v]))
        return dict(n_c=v[0].value, Kc=v[1].value, nout=v[2].value, b1s1=v[3].value, b1s2=v[4].value,
                    mask_bytes=v[5].value, c_chunk=v[6].value, t_chunk=v[7].value)

    def rotations(self):
        n = _u32()
        _check(lib().blb_cc_plan_rotations(self.h, None, 0, ctypes.byref(n)))
        out = (_i32 * max(1, n.value))()
        _check(lib().blb_cc_plan_rotations(self.h, out, n.value, ctypes.byref(n)))
        return list(out)[:n.value]


class Context:
    """blb_ctx: one parameter set on one CUDA stream (a torch stream; default:
    torch's current stream)."""

    def __init__(self, logN, q_bits, p_bits, dnum, scale=2.0 ** 40, stream=None, torch_allocator=True):
        import torch
        if torch_allocator:
            use_torch_allocator()
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        p, keep = _params(logN, q_bits, p_bits, dnum, scale)
        h = ctypes.c_void_p()
        _check(lib().blb_ctx_create(ctypes.byref(p), ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)))
        self.h = h.value
        self.logN, self.N, self.nQ, self.nP, self.dnum = logN, 1 << logN, len(q_bits), len(p_bits), dnum
        self.scale = scale
        out = np.zeros(self.nQ + self.nP, np.uint64)
        _check(lib().blb_ctx_primes(self.h, out.ctypes.data))
        self.primes = [int(x) for x in out]

    def free(self):
        if getattr(self, "h", None):
            lib().blb_ctx_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def _new(self, cls, fn, *args):
        h = ctypes.c_void_p()
        _check(fn(self.h, *args, ctypes.byref(h)))
        return cls(self, h.value)

    def key_bytes(self):
        """Device bytes of one switching key: dnum x 2 x (nQ + nP) x N words."""
        return self.dnum * 2 * (self.nQ + self.nP) * self.N * 8

    def sync(self):
        _check(lib().blb_ctx_sync(self.h))

    def bytes_in_use(self):
        return int(lib().blb_ctx_bytes_in_use(self.h))

    def set_wait_limit(self, limit_ns):
        """Limit of the bounded device waits in nanoseconds (0 = 2 s)."""
        _check(lib().blb_ctx_set_wait_limit(self.h, _u64(limit_ns)))

    def set_deferred_encode_check(self, on=True):
        """Encodings stop waiting for their overflow check; sync() raises if
        any encoding since the last sync overflowed."""
        _check(lib().blb_ctx_set_deferred_encode_check(self.h, int(on)))

    def set_batch_mac(self, kind):
        """MAC kernel of batched products: 0 automatic, 1 mma.sync, 2 tcgen05."""
        _check(lib().blb_ctx_set_batch_mac(self.h, int(kind)))

    def test_withhold_copies(self, withhold):
        """Test hook: the matmul_cp copy stage issues nothing, so waits expire."""
        _check(lib().blb_ctx_test_withhold_copies(self.h, int(withhold)))

    # keys
    def keygen(self, seed, rot_steps=(), relin=False):
        r = (_i32 * max(1, len(rot_steps)))(*rot_steps)
        return self._new(Keys, lib().blb_keygen, _u64(seed), r, len(rot_steps), int(relin))

    def keys_export(self, keys, which, rot=0):
        if which == 0:
            out = np.zeros(self.N, np.int64)
        else:
            out = np.zeros((self.dnum, 2, self.nQ + self.nP, self.N), np.uint64)
        _check(lib().blb_keys_export(self.h, keys.h, which, rot, out.ctypes.data))
        return out

    # encoding
    def encode(self, vals, level, scale=None):
        scale = self.scale if scale is None else scale
        if isinstance(vals, np.ndarray):
            vals = np.ascontiguousarray(vals, np.float64)
        n = int(vals.numel() if hasattr(vals, "numel") else vals.size)
        return self._new(Plaintext, lib().blb_encode, _ptr(vals), _u64(n), level, _dbl(scale))

    def encode_batch(self, vals, level, scale=None):
        """vals: (count, n) host array or device tensor -> list of count plaintexts."""
        scale = self.scale if scale is None else scale
        if isinstance(vals, np.ndarray):
            vals = np.ascontiguousarray(vals, np.float64)
        count, n = int(vals.shape[0]), int(vals.shape[1])
        out = (ctypes.c_void_p * count)()
        _check(lib().blb_encode_batch(self.h, _ptr(vals), _u64(n), count, level, _dbl(scale), out))
        return [Plaintext(self, p) for p in out]

    def pt_export(self, pt, level):
        out = np.zeros((level + 1, self.N), np.uint64)
        _check(lib().blb_pt_export(self.h, pt.h, out.ctypes.data))
        return out

    # ciphertexts
    def encrypt(self, keys, pt, nonce):
        return self._new(Ciphertext, lib().blb_encrypt, keys.h, pt.h, _u64(nonce))

    def encrypt_batch(self, keys, pts, nonces):
        count = len(pts)
        ps = (ctypes.c_void_p * count)(*[p.h for p in pts])
        ns = np.ascontiguousarray(nonces, np.uint64)
        out = (ctypes.c_void_p * count)()
        _check(lib().blb_encrypt_batch(self.h, keys.h, ps, count, ns.ctypes.data, out))
        return [Ciphertext(self, c) for c in out]

    def ct_export(self, ct, out=None):
        lv, npl, _ = ct.info()
        if out is None:
            out = np.zeros((npl, lv + 1, self.N), np.uint64)
        _check(lib().blb_ct_export(self.h, ct.h, _ptr(out)))
        return out

    def ct_import(self, coeffs, scale):
        coeffs = np.ascontiguousarray(coeffs, np.uint64) if isinstance(coeffs, np.ndarray) else coeffs
        npl, n = coeffs.shape[0], coeffs.shape[1]
        return self._new(Ciphertext, lib().blb_ct_import, _ptr(coeffs), n - 1, npl, _dbl(scale))

    def decrypt(self, keys, ct, coeffs=True, slots=True, coeff_out=None, slot_out=None):
        lv = ct.level
        if coeffs and coeff_out is None:
            coeff_out = np.zeros((lv + 1, self.N), np.uint64)
        if slots and slot_out is None:
            slot_out = np.zeros(self.N // 2, np.float64)
        _check(lib().blb_decrypt(self.h, keys.h, ct.h, _ptr(coeff_out) if coeffs else None,
                                 _ptr(slot_out) if slots else None))
        return coeff_out, slot_out

    def decrypt_batch(self, keys, cts, coeff_out=None, slot_out=None, coeffs=True, slots=False):
        """Ciphertexts of one level: coefficients (count, level+1, N), slots (count, N/2)."""
        count, lv = len(cts), cts[0].level
        if coeffs and coeff_out is None:
            coeff_out = np.zeros((count, lv + 1, self.N), np.uint64)
        if slots and slot_out is None:
            slot_out = np.zeros((count, self.N // 2), np.float64)
        cs = (ctypes.c_void_p * count)(*[c.h for c in cts])
        _check(lib().blb_decrypt_batch(self.h, keys.h, cs, count, _ptr(coeff_out) if coeffs else None,
                                       _ptr(slot_out) if slots else None))
        return coeff_out, slot_out

    # operations
    def rotate(self, keys, ct, steps):
        return self._new(Ciphertext, lib().blb_rotate, keys.h, ct.h, _i32(steps))

    def rescale(self, ct):
        _check(lib().blb_rescale(self.h, ct.h))
        return ct

    def add(self, a, b):
        return self._new(Ciphertext, lib().blb_add, a.h, b.h)

    def ct_copy(self, dst, src):
        _check(lib().blb_ct_copy(self.h, dst.h, src.h))

    def capture(self, fn, warmup=True):
        """Run fn once (sizing the library's arenas), then capture it into a
        CUDA graph on the context's stream; PyTorch's graph-private pool serves
        the library's allocations.  Returns (graph, fn's result): graph.replay()
        reruns every kernel on the same buffers, so the ciphertexts fn returned
        hold the latest replay's result (keep them alive with the graph)."""
        import torch
        if self.stream == torch.cuda.default_stream(self.stream.device):
            raise ValueError("graph capture needs a context created on a non-default stream")
        if warmup:
            fn()
            self.sync()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=self.stream, capture_error_mode="relaxed"):
            out = fn()
        return g, out

    def add_plain(self, a, pt):
        return self._new(Ciphertext, lib().blb_add_plain, a.h, pt.h)

    def pt_import(self, coeffs, level, scale=None):
        """Plaintext from (level+1, N) residues in coefficient form (host or device)."""
        scale = self.scale if scale is None else scale
        if isinstance(coeffs, np.ndarray):
            coeffs = np.ascontiguousarray(coeffs, np.uint64)
        return self._new(Plaintext, lib().blb_pt_import, _ptr(coeffs), level, _dbl(scale))

    # -- rotate-and-sum packing (Sec. 4.2.1) and the LayerNorm head ----------
    def rotate_sum_packing(self, keys, cts, L, D, direction=0, mask=False):
        count = len(cts)
        ins = (ctypes.c_void_p * count)(*[c.h for c in cts])
        out = (ctypes.c_void_p * count)()
        _check(lib().blb_rotate_sum_packing(self.h, keys.h, ins, count, L, D, int(direction), int(mask), out))
        return [Ciphertext(self, c) for c in out]

    def layernorm_head(self, keys, X, L, D, nc):
        """X: count sequences x nc ciphertexts (flat list, sequence-major).
        Returns (X_mu as a flat list, var one per sequence)."""
        total = len(X)
        if total % nc:
            raise ValueError("X must hold nc ciphertexts per sequence")
        count = total // nc
        ins = (ctypes.c_void_p * total)(*[c.h for c in X])
        xm = (ctypes.c_void_p * total)()
        var = (ctypes.c_void_p * count)()
        _check(lib().blb_layernorm_head(self.h, keys.h, ins, count, nc, L, D, xm, var))
        return [Ciphertext(self, c) for c in xm], [Ciphertext(self, c) for c in var]

    # -- local steps of the conversions (Alg. 1 steps 3-4, Alg. 2, App. C.3) --
    # 128-bit shares are (..., 2) uint64 arrays (low, high); every array may be
    # a numpy array or a torch tensor (host or device).
    @staticmethod
    def _count(a, per):
        n = int(a.numel() if hasattr(a, "numel") else np.asarray(a).size)
        if n % per:
            raise ValueError(f"array of {n} words is not a whole number of {per}-word members")
        return n // per

    @staticmethod
    def _c(a):
        return np.ascontiguousarray(a, np.uint64) if isinstance(a, np.ndarray) else a

    def f2r_wrap_sim(self, t0, t1, seed, nonces, w0=None, w1=None):
        t0, t1 = self._c(t0), self._c(t1)
        count = self._count(t0, self.N)
        w0 = np.zeros((count, self.N, 2), np.uint64) if w0 is None else w0
        w1 = np.zeros((count, self.N, 2), np.uint64) if w1 is None else w1
        ns = np.ascontiguousarray(nonces, np.uint64).reshape(-1)
        assert len(ns) == count
        _check(lib().blb_f2r_wrap_sim(self.h, _ptr(t0), _ptr(t1), count, _u64(seed), ns.ctypes.data,
                                      _ptr(w0), _ptr(w1)))
        return w0, w1

    def c2m_local(self, party, t, wsh, scale, l=43, sf=13, out=None):
        t, wsh = self._c(t), self._c(wsh)
        count = self._count(t, self.N)
        out = np.zeros((count, self.N // 2), np.uint64) if out is None else out
        _check(lib().blb_c2m_local(self.h, party, _ptr(t), _ptr(wsh), count, _dbl(scale), l, sf, _ptr(out)))
        return out

    def ext_wrap_sim(self, x0, x1, n, l, seed, nonces, w0=None, w1=None):
        x0, x1 = self._c(x0), self._c(x1)
        count = self._count(x0, n) if n else len(nonces)
        w0 = np.zeros((count, n, 2), np.uint64) if w0 is None else w0
        w1 = np.zeros((count, n, 2), np.uint64) if w1 is None else w1
        ns = np.ascontiguousarray(nonces, np.uint64).reshape(-1)
        assert len(ns) == count
        _check(lib().blb_ext_wrap_sim(self.h, _ptr(x0), _ptr(x1), n, count, l, _u64(seed), ns.ctypes.data,
                                      _ptr(w0), _ptr(w1)))
        return w0, w1

    def m2c_local(self, party, x, wsh, n, level, scale, l=43, sf=13, count=None, out=None):
        x, wsh = self._c(x), self._c(wsh)
        count = (self._count(x, n) if n else 1) if count is None else count
        out = np.zeros((count, level + 1, self.N), np.uint64) if out is None else out
        _check(lib().blb_m2c_local(self.h, party, _ptr(x), _ptr(wsh), n, count, level, _dbl(scale), l, sf,
                                   _ptr(out)))
        return out

    def sub(self, a, b):
        return self._new(Ciphertext, lib().blb_sub, a.h, b.h)

    def drop_level(self, a, level):
        return self._new(Ciphertext, lib().blb_drop_level, a.h, level)

    def mul_const(self, a, vals, target_scale=None):
        """a times the slot vector vals (a scalar broadcasts), rescaled to
        target_scale (default: a's scale)."""
        v = np.ascontiguousarray(np.atleast_1d(vals), np.float64)
        ts = a.scale if target_scale is None else target_scale
        return self._new(Ciphertext, lib().blb_mul_const, a.h, v.ctypes.data, _u64(len(v)), _dbl(ts))

    def mul_plain(self, a, pt):
        return self._new(Ciphertext, lib().blb_mul_plain, a.h, pt.h)

    def mul(self, keys, a, b, relin=True):
        return self._new(Ciphertext, lib().blb_mul, keys.h if keys else None, a.h, b.h, int(relin))

    def relinearize(self, keys, ct):
        return self._new(Ciphertext, lib().blb_relinearize, keys.h, ct.h)

    def keyswitch_coeffs(self, keys, rot, d):
        d = np.ascontiguousarray(d, np.uint64)
        n = d.shape[0]
        out = np.zeros((2, n, self.N), np.uint64)
        _check(lib().blb_keyswitch_coeffs(self.h, keys.h, _i32(rot), d.ctypes.data, n - 1, out.ctypes.data))
        return out

    def keyswitch_noalloc(self, keys, rot, d, out):
        """Allocation-free key switch (blb_keyswitch_noalloc): d is (level+1, N)
        and out (2, level+1, N), host numpy arrays or device tensors."""
        n = d.shape[0]
        _check(lib().blb_keyswitch_noalloc(self.h, keys.h, _i32(rot), _ptr(d), n - 1, _ptr(out)))
        return out

    # matmul_cp
    def cp_plan(self, m, d, W, d_out, level, b1=0):
        if isinstance(W, np.ndarray):
            W = np.ascontiguousarray(W, np.float64)
        s = _Sched(b1)
        return self._new(CpPlan, lib().blb_cp_plan_create, m, d, _ptr(W), d_out, level, ctypes.byref(s))

    def cp_plan_diag(self, L, groups, Dh, W, d_out, level, b1=0):
        """Diagonal-input plan (App. C.2): groups = heads per head group."""
        W = np.ascontiguousarray(W, np.float64) if isinstance(W, np.ndarray) else W
        hg = np.ascontiguousarray(groups, np.uint32)
        s = _Sched(b1)
        return self._new(CpPlan, lib().blb_cp_plan_create_diag, L, len(groups), hg.ctypes.data, Dh, _ptr(W), d_out,
                         level, ctypes.byref(s))

    def matmul_cp_plan(self, keys, plan, X):
        info = plan.info()
        xs = (ctypes.c_void_p * len(X))(*[x.h for x in X])
        ys = (ctypes.c_void_p * info["nY"])()
        _check(lib().blb_matmul_cp_plan(self.h, keys.h, plan.h, xs, len(X), ys))
        return [Ciphertext(self, y) for y in ys]

    def matmul_cp_batch(self, keys, plan, X_seqs):
        """X_seqs: list of per-sequence lists of nX ciphertexts -> list of lists of nY."""
        info = plan.info()
        flat = [x for seq in X_seqs for x in seq]
        xs = (ctypes.c_void_p * len(flat))(*[x.h for x in flat])
        ys = (ctypes.c_void_p * (len(X_seqs) * info["nY"]))()
        _check(lib().blb_matmul_cp_batch(self.h, keys.h, plan.h, xs, len(X_seqs), ys))
        out = [Ciphertext(self, y) for y in ys]
        return [out[s * info["nY"]:(s + 1) * info["nY"]] for s in range(len(X_seqs))]

    def matmul_cp_multi(self, keys_list, plan, X_seqs):
        """One key set per sequence (different clients) -> list of lists of nY."""
        info = plan.info()
        flat = [x for seq in X_seqs for x in seq]
        xs = (ctypes.c_void_p * len(flat))(*[x.h for x in flat])
        ks = (ctypes.c_void_p * len(keys_list))(*[k.h for k in keys_list])
        ys = (ctypes.c_void_p * (len(X_seqs) * info["nY"]))()
        _check(lib().blb_matmul_cp_multi(self.h, ks, plan.h, xs, len(X_seqs), ys))
        out = [Ciphertext(self, y) for y in ys]
        return [out[s * info["nY"]:(s + 1) * info["nY"]] for s in range(len(X_seqs))]

    def matmul_cp(self, keys, X, m, d, W, d_out, b1=0):
        W = np.ascontiguousarray(W, np.float64) if isinstance(W, np.ndarray) else W
        k = (self.N // 2) // m
        nY = (d_out + k - 1) // k
        xs = (ctypes.c_void_p * len(X))(*[x.h for x in X])
        ys = (ctypes.c_void_p * nY)()
        s = _Sched(b1)
        _check(lib().blb_matmul_cp(self.h, keys.h, xs, len(X), m, d, _ptr(W), d_out, ctypes.byref(s), ys))
        return [Ciphertext(self, y) for y in ys]

    # matmul_cc
    def cc_plan(self, L, Hg, R, level, b1s1=0, b1s2=0, c_chunk=0, t_chunk=0, workspace_bytes=0):
        s = _CcSched(b1s1, b1s2, c_chunk, t_chunk, workspace_bytes)
        return self._new(CcPlan, lib().blb_cc_plan_create, L, Hg, R, level, ctypes.byref(s))

    def matmul_cc_plan(self, keys, plan, A, B):
        info = plan.info()
        a = (ctypes.c_void_p * len(A))(*[x.h for x in A])
        b = (ctypes.c_void_p * len(B))(*[x.h for x in B])
        out = (ctypes.c_void_p * info["nout"])()
        _check(lib().blb_matmul_cc_plan(self.h, keys.h, plan.h, a, b, len(A), out))
        return [Ciphertext(self, y) for y in out]

    # CKKS -> MPC
    def he2mpc(self, keys, ct, nonce, share_out=None):
        if share_out is None:
            share_out = np.zeros(self.N, np.uint64)
        h = ctypes.c_void_p()
        _check(lib().blb_he2mpc(self.h, keys.h, ct.h, _u64(nonce), ctypes.byref(h), _ptr(share_out)))
        return Ciphertext(self, h.value), share_out

    def he2mpc_batch(self, keys, cts, nonces, share_out=None):
        count = len(cts)
        if share_out is None:
            share_out = np.zeros((count, self.N), np.uint64)
        cs = (ctypes.c_void_p * count)(*[c.h for c in cts])
        ns = np.ascontiguousarray(nonces, np.uint64)
        out = (ctypes.c_void_p * count)()
        _check(lib().blb_he2mpc_batch(self.h, keys.h, cs, count, ns.ctypes.data, out, _ptr(share_out)))
        return [Ciphertext(self, c) for c in out], share_out

    def profile(self, on=True, only=None):
        """Enable (and reset) the per-site CUDA-event profile; only: one site name."""
        _check(lib().blb_profile_enable(self.h, int(on)))
        _check(lib().blb_profile_select(self.h, only.encode() if only else None))

    def profile_read(self, site):
        ms, cnt, nb = _dbl(), _u64(), _u64()
        _check(lib().blb_profile_read(self.h, site.encode(), ctypes.byref(ms), ctypes.byref(cnt), ctypes.byref(nb)))
        return ms.value, cnt.value, nb.value

    def profile_read_ops(self, site):
        """(128-bit multiply-adds, 128-bit reductions, butterflies) counted at a site."""
        m, r, b = _u64(), _u64(), _u64()
        _check(lib().blb_profile_read_ops(self.h, site.encode(), ctypes.byref(m), ctypes.byref(r), ctypes.byref(b)))
        return m.value, r.value, b.value

    def ntt_autotune(self, rows=64):
        """Time the NTT's radices (8, 16) and pass splits (-1, 0, +1); keep
        the fastest pair.  Returns (split, radix, {(radix, split):
        microseconds per row and direction})."""
        sp, rx, us = ctypes.c_int(), ctypes.c_int(), (_dbl * 6)()
        _check(lib().blb_ntt_autotune(self.h, rows, ctypes.byref(sp), ctypes.byref(rx), us))
        return sp.value, rx.value, {((8, 16)[k // 3], k % 3 - 1): us[k] for k in range(6) if us[k] > 0}

    def ntt_set_split(self, split):
        _check(lib().blb_ntt_set_split(self.h, int(split)))

    def ntt_set_radix(self, radix):
        _check(lib().blb_ntt_set_radix(self.h, int(radix)))

    def ntt(self, data, prime_idx, inverse=False):
        data = np.ascontiguousarray(data, np.uint64).copy()
        pi = np.ascontiguousarray(prime_idx, np.uint32)
        _check(lib().blb_ntt(self.h, data.ctypes.data, data.shape[0], pi.ctypes.data, int(inverse)))
        return data
