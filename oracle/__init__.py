"""CPU oracle of BLB's RNS-CKKS linear path (arXiv 2508.19525).

TEST INFRASTRUCTURE ONLY: imported by the test suite, the smoke check and the
benchmark's CPU-baseline leg, never by the product library.  This wrapper only
marshals numpy arrays into the C oracle (oracle.c); every operation is computed
there.
"""
import ctypes
import numpy as np

from .build import build

_u64p = ctypes.POINTER(ctypes.c_uint64)
_i64p = ctypes.POINTER(ctypes.c_int64)
_f64p = ctypes.POINTER(ctypes.c_double)
_u32p = ctypes.POINTER(ctypes.c_uint32)

MAX_PRIMES = 32
SECRET, KEY_A, KEY_E, ENC_A, ENC_E, MASK, WRAP = 1, 2, 3, 4, 5, 6, 7
FX_F, FX_P = 30, 26  # fraction bits of the share-FFT roots; resolution of its data


class _Params(ctypes.Structure):
    _fields_ = [("logN", ctypes.c_uint32), ("N", ctypes.c_uint32), ("nQ", ctypes.c_uint32),
                ("nP", ctypes.c_uint32), ("dnum", ctypes.c_uint32), ("alpha", ctypes.c_uint32),
                ("prime", ctypes.c_uint64 * MAX_PRIMES), ("psi", ctypes.c_uint64 * MAX_PRIMES)]


class _GaloisSet(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint32), ("gal", _u64p), ("ksk", ctypes.POINTER(_u64p))]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        L = _lib
        L.orc_galois_elt.restype = ctypes.c_uint64
        L.orc_ksk_words.restype = ctypes.c_uint64
        L.orc_cp_num_rotations.restype = ctypes.c_uint32
        L.orc_cc_num_rotations.restype = ctypes.c_uint32
        L.orc_is_prime.argtypes = [ctypes.c_uint64]
        L.orc_galois_elt.argtypes = [ctypes.c_void_p, ctypes.c_int32]
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def philox(ctr, key):
    c = (ctypes.c_uint32 * 4)(*ctr)
    k = (ctypes.c_uint32 * 2)(*key)
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox(c, k, o)
    return list(o)


def u128_words(vals):
    """Python ints (any sign) -> (n, 2) uint64 words of their residues mod 2^128."""
    v = [int(x) % (1 << 128) for x in vals]
    return np.array([[x & (2**64 - 1), x >> 64] for x in v], np.uint64).reshape(len(v), 2)


def words_u128(w):
    """(n, 2) uint64 words -> Python ints in [0, 2^128)."""
    w = np.asarray(w, np.uint64).reshape(-1, 2)
    return [int(a) | (int(b) << 64) for a, b in w]


def share_trunc(party, x, k):
    """Party's local truncation of 128-bit shares ((n, 2) words) by k bits."""
    x = np.ascontiguousarray(x, np.uint64).reshape(-1, 2)
    out = np.zeros_like(x)
    lib().orc_share_trunc(party, _p(x, _u64p), ctypes.c_uint64(len(x)), k, _p(out, _u64p))
    return out


def f2r_wrap_sim(q, t0, t1, seed, nonce):
    t0 = np.ascontiguousarray(t0, np.uint64)
    t1 = np.ascontiguousarray(t1, np.uint64)
    w0, w1 = np.zeros((len(t0), 2), np.uint64), np.zeros((len(t0), 2), np.uint64)
    lib().orc_f2r_wrap_sim(len(t0), ctypes.c_uint64(q), _p(t0, _u64p), _p(t1, _u64p), ctypes.c_uint64(seed),
                           nonce, _p(w0, _u64p), _p(w1, _u64p))
    return w0, w1


def f2r_local(party, q, t, wsh):
    t = np.ascontiguousarray(t, np.uint64)
    wsh = np.ascontiguousarray(wsh, np.uint64)
    U = np.zeros((len(t), 2), np.uint64)
    lib().orc_f2r_local(party, len(t), ctypes.c_uint64(q), _p(t, _u64p), _p(wsh, _u64p), _p(U, _u64p))
    return U


def ext_wrap_sim(l, x0, x1, seed, nonce):
    x0 = np.ascontiguousarray(x0, np.uint64)
    x1 = np.ascontiguousarray(x1, np.uint64)
    w0, w1 = np.zeros((len(x0), 2), np.uint64), np.zeros((len(x0), 2), np.uint64)
    lib().orc_ext_wrap_sim(len(x0), l, _p(x0, _u64p), _p(x1, _u64p), ctypes.c_uint64(seed), nonce,
                           _p(w0, _u64p), _p(w1, _u64p))
    return w0, w1


def ext_local(party, l, x, wsh):
    x = np.ascontiguousarray(x, np.uint64)
    wsh = np.ascontiguousarray(wsh, np.uint64)
    X = np.zeros((len(x), 2), np.uint64)
    lib().orc_ext_local(party, len(x), l, _p(x, _u64p), _p(wsh, _u64p), _p(X, _u64p))
    return X


def is_prime(n):
    return bool(lib().orc_is_prime(ctypes.c_uint64(n)))


def cdt_table():
    t = np.zeros(19, np.uint64)
    lib().orc_cdt_table(_p(t, _u64p))
    return t


def sample_ternary(N, seed, obj, purpose, j=0):
    out = np.zeros(N, np.int64)
    lib().orc_sample_ternary(ctypes.c_uint32(N), ctypes.c_uint64(seed), ctypes.c_uint32(obj),
                             ctypes.c_uint32(purpose), ctypes.c_uint32(j), _p(out, _i64p))
    return out


def sample_gauss(N, seed, obj, purpose, j=0):
    out = np.zeros(N, np.int64)
    lib().orc_sample_gauss(ctypes.c_uint32(N), ctypes.c_uint64(seed), ctypes.c_uint32(obj),
                           ctypes.c_uint32(purpose), ctypes.c_uint32(j), _p(out, _i64p))
    return out


def sample_uniform(N, q, seed, obj, purpose, j=0):
    out = np.zeros(N, np.uint64)
    lib().orc_sample_uniform(ctypes.c_uint32(N), ctypes.c_uint64(q), ctypes.c_uint64(seed),
                             ctypes.c_uint32(obj), ctypes.c_uint32(purpose), ctypes.c_uint32(j),
                             _p(out, _u64p))
    return out


class Oracle:
    """One parameter set.  Polynomials are numpy uint64 arrays in coefficient
    form, shape (..., limbs, N); ciphertexts have shape (polys, level+1, N)."""

    def __init__(self, logN, q_bits, p_bits, dnum):
        self.P = _Params()
        qb = (ctypes.c_uint32 * len(q_bits))(*q_bits)
        pb = (ctypes.c_uint32 * len(p_bits))(*p_bits)
        rc = lib().orc_params_init(ctypes.byref(self.P), logN, len(q_bits), len(p_bits), qb, pb, dnum)
        if rc:
            raise ValueError(f"orc_params_init failed: {rc}")
        self.logN, self.N = logN, 1 << logN
        self.nQ, self.nP, self.dnum, self.alpha = len(q_bits), len(p_bits), dnum, self.P.alpha
        self.primes = [int(self.P.prime[i]) for i in range(self.nQ + self.nP)]
        self.psi = [int(self.P.psi[i]) for i in range(self.nQ + self.nP)]
        self._pp = ctypes.byref(self.P)

    # -- ring --------------------------------------------------------------
    def galois_elt(self, r):
        return int(lib().orc_galois_elt(self._pp, r))

    def ntt(self, a, prime_idx):
        a = np.ascontiguousarray(a, np.uint64).copy()
        lib().orc_ntt(self._pp, prime_idx, _p(a, _u64p))
        return a

    def intt(self, a, prime_idx):
        a = np.ascontiguousarray(a, np.uint64).copy()
        lib().orc_intt(self._pp, prime_idx, _p(a, _u64p))
        return a

    def negacyclic_mul(self, a, b, prime_idx):
        a = np.ascontiguousarray(a, np.uint64)
        b = np.ascontiguousarray(b, np.uint64)
        out = np.zeros(self.N, np.uint64)
        lib().orc_negacyclic_mul(self._pp, prime_idx, _p(a, _u64p), _p(b, _u64p), _p(out, _u64p))
        return out

    # -- encoding ----------------------------------------------------------
    def encode_int(self, z, scale):
        z = np.ascontiguousarray(z, np.float64)
        out = np.zeros(self.N, np.int64)
        rc = lib().orc_encode_int(self._pp, _p(z, _f64p), len(z), ctypes.c_double(scale), _p(out, _i64p))
        if rc:
            raise ValueError(f"encode failed {rc}")
        return out

    def encode(self, z, level, scale):
        z = np.ascontiguousarray(z, np.float64)
        out = np.zeros((level + 1, self.N), np.uint64)
        rc = lib().orc_encode(self._pp, _p(z, _f64p), len(z), level, ctypes.c_double(scale), _p(out, _u64p))
        if rc:
            raise ValueError(f"encode failed {rc}")
        return out

    def decode(self, coef, scale):
        coef = np.ascontiguousarray(coef, np.int64)
        z = np.zeros(self.N // 2, np.float64)
        lib().orc_decode(self._pp, _p(coef, _i64p), ctypes.c_double(scale), _p(z, _f64p))
        return z

    def centered(self, limb, prime_idx=0):
        q = self.primes[prime_idx]
        v = np.asarray(limb, np.uint64)
        return np.where(v > q // 2, -(np.uint64(q) - v).astype(np.int64), v.astype(np.int64))

    # -- keys --------------------------------------------------------------
    def ksk_shape(self):
        return (self.dnum, 2, self.nQ + self.nP, self.N)

    def keygen_secret(self, seed):
        s = np.zeros(self.N, np.int64)
        lib().orc_keygen_secret(self._pp, ctypes.c_uint64(seed), _p(s, _i64p))
        return s

    def keygen_relin(self, seed, s):
        k = np.zeros(self.ksk_shape(), np.uint64)
        lib().orc_keygen_relin(self._pp, ctypes.c_uint64(seed), _p(s, _i64p), _p(k, _u64p))
        return k

    def keygen_galois(self, seed, s, g):
        k = np.zeros(self.ksk_shape(), np.uint64)
        lib().orc_keygen_galois(self._pp, ctypes.c_uint64(seed), _p(s, _i64p), ctypes.c_uint64(g), _p(k, _u64p))
        return k

    def keygen_ksk(self, seed, s, s_prime, obj):
        k = np.zeros(self.ksk_shape(), np.uint64)
        s_prime = np.ascontiguousarray(s_prime, np.int64)
        lib().orc_keygen_ksk(self._pp, ctypes.c_uint64(seed), _p(s, _i64p), _p(s_prime, _i64p), obj, _p(k, _u64p))
        return k

    # -- ciphertexts -------------------------------------------------------
    def encrypt(self, s, pt, seed, nonce):
        pt = np.ascontiguousarray(pt, np.uint64)
        level = pt.shape[0] - 1
        ct = np.zeros((2, level + 1, self.N), np.uint64)
        lib().orc_encrypt(self._pp, _p(s, _i64p), _p(pt, _u64p), level, ctypes.c_uint64(seed), nonce, _p(ct, _u64p))
        return ct

    def decrypt(self, s, ct):
        ct = np.ascontiguousarray(ct, np.uint64)
        npolys, n = ct.shape[0], ct.shape[1]
        m = np.zeros((n, self.N), np.uint64)
        lib().orc_decrypt(self._pp, _p(s, _i64p), _p(ct, _u64p), n - 1, npolys, _p(m, _u64p))
        return m

    def automorphism(self, poly, g):
        poly = np.ascontiguousarray(poly, np.uint64)
        out = np.zeros_like(poly)
        lib().orc_automorphism(self._pp, _p(poly, _u64p), poly.shape[0], ctypes.c_uint64(g), _p(out, _u64p))
        return out

    def keyswitch(self, d, ksk):
        d = np.ascontiguousarray(d, np.uint64)
        n = d.shape[0]
        out = np.zeros((2, n, self.N), np.uint64)
        lib().orc_keyswitch(self._pp, _p(d, _u64p), n - 1, _p(np.ascontiguousarray(ksk), _u64p), _p(out, _u64p))
        return out

    def moddown(self, acc, level):
        """acc: (2, level+1+nP, N) over Q_l then P -> (2, level+1, N)."""
        acc = np.ascontiguousarray(acc, np.uint64)
        out = np.zeros((2, level + 1, self.N), np.uint64)
        lib().orc_moddown(self._pp, _p(acc, _u64p), level, _p(out, _u64p))
        return out

    def rotate(self, ct, r, gksk):
        ct = np.ascontiguousarray(ct, np.uint64)
        out = np.zeros_like(ct)
        lib().orc_rotate(self._pp, _p(ct, _u64p), ct.shape[1] - 1, r, _p(np.ascontiguousarray(gksk), _u64p), _p(out, _u64p))
        return out

    def rotate_hoisted(self, ct, rots, gksks):
        """Rotations of one ciphertext sharing one ModUp: list of (2, n, N)."""
        ct = np.ascontiguousarray(ct, np.uint64)
        k = len(rots)
        out = np.zeros((k,) + ct.shape, np.uint64)
        keys = [np.ascontiguousarray(x, np.uint64) for x in gksks]
        kp = (ctypes.POINTER(ctypes.c_uint64) * max(k, 1))(*[_p(x, _u64p) for x in keys])
        r = (ctypes.c_int32 * max(k, 1))(*rots)
        lib().orc_rotate_hoisted(self._pp, _p(ct, _u64p), ct.shape[1] - 1, k, r, kp, _p(out, _u64p))
        return list(out)

    def rotate_sum(self, base, Ts, rots, gksks):
        """base + sum_x Rot^{rots[x]}(Ts[x]) with one ModDown; base may be None."""
        k = len(Ts)
        shape = np.shape(base) if k == 0 else np.shape(Ts[0])
        Ts = np.ascontiguousarray(np.stack(Ts) if k else np.zeros((1,) + tuple(shape)), np.uint64)
        out = np.zeros(shape, np.uint64)
        keys = [np.ascontiguousarray(x, np.uint64) for x in gksks]
        kp = (ctypes.POINTER(ctypes.c_uint64) * max(k, 1))(*[_p(x, _u64p) for x in keys])
        r = (ctypes.c_int32 * max(k, 1))(*rots)
        bp = None if base is None else np.ascontiguousarray(base, np.uint64)
        lib().orc_rotate_sum(self._pp, None if bp is None else _p(bp, _u64p), _p(Ts, _u64p), shape[1] - 1, k, r, kp,
                             _p(out, _u64p))
        return out

    def rescale(self, ct):
        ct = np.ascontiguousarray(ct, np.uint64)
        npolys, n = ct.shape[0], ct.shape[1]
        out = np.zeros((npolys, n - 1, self.N), np.uint64)
        lib().orc_rescale(self._pp, _p(ct, _u64p), n - 1, npolys, _p(out, _u64p))
        return out

    def mul_plain(self, ct, pt):
        ct = np.ascontiguousarray(ct, np.uint64)
        out = np.zeros_like(ct)
        lib().orc_mul_plain(self._pp, _p(ct, _u64p), _p(np.ascontiguousarray(pt, np.uint64), _u64p), ct.shape[1] - 1, _p(out, _u64p))
        return out

    def tensor(self, a, b):
        a = np.ascontiguousarray(a, np.uint64)
        b = np.ascontiguousarray(b, np.uint64)
        out = np.zeros((3,) + a.shape[1:], np.uint64)
        lib().orc_tensor(self._pp, _p(a, _u64p), _p(b, _u64p), a.shape[1] - 1, _p(out, _u64p))
        return out

    def relinearize(self, ct3, rksk):
        ct3 = np.ascontiguousarray(ct3, np.uint64)
        out = np.zeros((2,) + ct3.shape[1:], np.uint64)
        lib().orc_relinearize(self._pp, _p(ct3, _u64p), ct3.shape[1] - 1, _p(np.ascontiguousarray(rksk), _u64p), _p(out, _u64p))
        return out

    # -- protocols ---------------------------------------------------------
    def matmul_cp(self, X_cts, m, d, W, d_out, b1, galois, out_idx=None):
        """X_cts: (nX, 2, level+1, N); galois: dict g -> ksk array."""
        X_cts = np.ascontiguousarray(X_cts, np.uint64)
        nX, level = X_cts.shape[0], X_cts.shape[2] - 1
        k = (self.N // 2) // m
        nY = (d_out + k - 1) // k
        out_idx = list(range(nY)) if out_idx is None else list(out_idx)
        W = np.ascontiguousarray(W, np.float64)
        gals = np.array(list(galois.keys()), np.uint64)
        keys = [np.ascontiguousarray(galois[int(g)], np.uint64) for g in gals]
        ptrs = (_u64p * len(keys))(*[_p(kk, _u64p) for kk in keys])
        gs = _GaloisSet(len(keys), _p(gals, _u64p), ptrs)
        oi = np.array(out_idx, np.uint32)
        Y = np.zeros((len(out_idx), 2, level, self.N), np.uint64)
        rc = lib().orc_matmul_cp(self._pp, ctypes.byref(gs), _p(X_cts, _u64p), nX, level, m, d,
                                 _p(W, _f64p), d_out, b1, _p(oi, _u32p), len(out_idx), _p(Y, _u64p))
        if rc:
            raise ValueError(f"orc_matmul_cp failed: {rc}")
        return Y

    @staticmethod
    def _galois_set(galois):
        gals = np.array(list(galois.keys()), np.uint64)
        keys = [np.ascontiguousarray(galois[int(g)], np.uint64) for g in gals]
        ptrs = (_u64p * max(1, len(keys)))(*[_p(kk, _u64p) for kk in keys])
        return _GaloisSet(len(keys), _p(gals, _u64p), ptrs), (gals, keys, ptrs)

    def cp_baby_steps(self, X_cts, m, b1, galois):
        """The baby steps of matmul_cp: (nX, b1, 2, level+1, N), [c][b] = Rot^{b m}(X_c)."""
        X_cts = np.ascontiguousarray(X_cts, np.uint64)
        nX, level = X_cts.shape[0], X_cts.shape[2] - 1
        gs, _keep = self._galois_set(galois)
        baby = np.zeros((nX, b1, 2, level + 1, self.N), np.uint64)
        rc = lib().orc_cp_baby_steps(self._pp, ctypes.byref(gs), _p(X_cts, _u64p), nX, level, m, b1, _p(baby, _u64p))
        if rc:
            raise ValueError(f"orc_cp_baby_steps failed: {rc}")
        return baby

    def cp_encode_diagonals(self, level, m, d, W, d_out, b1, out_idx):
        """Plaintext diagonals of the given outputs: (n_out, G, nX, b1, level+1, N)."""
        k = (self.N // 2) // m
        G, nX = k // b1, (d + k - 1) // k
        W = np.ascontiguousarray(W, np.float64)
        oi = np.array(list(out_idx), np.uint32)
        pts = np.zeros((len(oi), G, nX, b1, level + 1, self.N), np.uint64)
        rc = lib().orc_cp_encode_diagonals(self._pp, level, m, d, _p(W, _f64p), d_out, b1, _p(oi, _u32p), len(oi),
                                           _p(pts, _u64p))
        if rc:
            raise ValueError(f"orc_cp_encode_diagonals failed: {rc}")
        return pts

    def cp_outputs(self, baby, m, b1, pts, galois):
        """Outputs of matmul_cp from its baby steps and pre-encoded plaintexts."""
        baby = np.ascontiguousarray(baby, np.uint64)
        pts = np.ascontiguousarray(pts, np.uint64)
        nX, level = baby.shape[0], baby.shape[3] - 1
        gs, _keep = self._galois_set(galois)
        Y = np.zeros((pts.shape[0], 2, level, self.N), np.uint64)
        rc = lib().orc_cp_outputs(self._pp, ctypes.byref(gs), _p(baby, _u64p), nX, level, m, b1, _p(pts, _u64p),
                                  pts.shape[0], _p(Y, _u64p))
        if rc:
            raise ValueError(f"orc_cp_outputs failed: {rc}")
        return Y

    def cp_inner_sum(self, baby, pts):
        """sum_c sum_b baby[c][b] (.) pts[c][b]: baby (nX, b1, 2, l+1, N), pts (nX, b1, l+1, N)."""
        baby = np.ascontiguousarray(baby, np.uint64)
        pts = np.ascontiguousarray(pts, np.uint64)
        nX, b1, level = baby.shape[0], baby.shape[1], baby.shape[3] - 1
        T = np.zeros((2, level + 1, self.N), np.uint64)
        rc = lib().orc_cp_inner_sum(self._pp, _p(baby, _u64p), nX, level, b1, _p(pts, _u64p), _p(T, _u64p))
        if rc:
            raise ValueError(f"orc_cp_inner_sum failed: {rc}")
        return T

    def matmul_cp_diag(self, X_cts, L, groups, Dh, W, d_out, b1, galois, out_idx=None):
        """Diagonal-input product (App. C.2).  X_cts: the dense-diagonal
        ciphertexts of every head group in order; groups: heads per group."""
        X_cts = np.ascontiguousarray(X_cts, np.uint64)
        level = X_cts.shape[2] - 1
        k = (self.N // 2) // L
        nY = (d_out + k - 1) // k
        out_idx = list(range(nY)) if out_idx is None else list(out_idx)
        W = np.ascontiguousarray(W, np.float64)
        hg = np.array(groups, np.uint32)
        gals = np.array(list(galois.keys()), np.uint64)
        keys = [np.ascontiguousarray(galois[int(g)], np.uint64) for g in gals]
        ptrs = (_u64p * max(1, len(keys)))(*[_p(kk, _u64p) for kk in keys])
        gs = _GaloisSet(len(keys), _p(gals, _u64p), ptrs)
        oi = np.array(out_idx, np.uint32)
        Y = np.zeros((len(out_idx), 2, level, self.N), np.uint64)
        rc = lib().orc_matmul_cp_diag(self._pp, ctypes.byref(gs), _p(X_cts, _u64p), level, L, len(groups),
                                      _p(hg, _u32p), Dh, _p(W, _f64p), d_out, b1, _p(oi, _u32p), len(out_idx),
                                      _p(Y, _u64p))
        if rc:
            raise ValueError(f"orc_matmul_cp_diag failed: {rc}")
        return Y

    def matmul_cc(self, A_cts, B_cts, L, Hg, b1s1, b1s2, galois, relin):
        """A_cts, B_cts: (n_c, 2, level+1, N) -> C: (L/Kc, 2, level-3, N)."""
        A_cts = np.ascontiguousarray(A_cts, np.uint64)
        B_cts = np.ascontiguousarray(B_cts, np.uint64)
        n_c, level = A_cts.shape[0], A_cts.shape[2] - 1
        Kc = (self.N // 2) // (L * Hg)
        gals = np.array(list(galois.keys()), np.uint64)
        keys = [np.ascontiguousarray(galois[int(g)], np.uint64) for g in gals]
        ptrs = (_u64p * max(1, len(keys)))(*[_p(kk, _u64p) for kk in keys])
        gs = _GaloisSet(len(keys), _p(gals, _u64p), ptrs)
        C = np.zeros((L // Kc, 2, level - 3, self.N), np.uint64)
        rc = lib().orc_matmul_cc(self._pp, ctypes.byref(gs), _p(np.ascontiguousarray(relin, np.uint64), _u64p),
                                 _p(A_cts, _u64p), _p(B_cts, _u64p), n_c, level, L, Hg, b1s1, b1s2, _p(C, _u64p))
        if rc:
            raise ValueError(f"orc_matmul_cc failed: {rc}")
        return C

    def cc_num_rotations(self, n_c, L, Kc, b1s1, b1s2):
        return int(lib().orc_cc_num_rotations(n_c, L, Kc, b1s1, b1s2))

    def cp_num_rotations(self, nX, nY, b1, G):
        return int(lib().orc_cp_num_rotations(nX, nY, b1, G))

    # -- rotate-and-sum packing (Sec. 4.2.1) and the LayerNorm head ------------
    def rs_packing(self, ct, L, D, direction, mask, gks):
        """gks: Galois keys of the rotations 2^i L (left, direction 0) or -2^i L (right)."""
        ct = np.ascontiguousarray(ct, np.uint64)
        level = ct.shape[1] - 1
        out = np.zeros((2, level + (0 if mask else 1), self.N), np.uint64)
        keys = [np.ascontiguousarray(k, np.uint64) for k in gks]
        arr = (_u64p * max(1, len(keys)))(*[_p(k, _u64p) for k in keys])
        rc = lib().orc_rs_packing(self._pp, _p(ct, _u64p), level, L, D, int(direction), int(mask), arr, _p(out, _u64p))
        if rc:
            raise ValueError(f"rs_packing failed {rc}")
        return out

    def layernorm_head(self, X_cts, L, D, gks, relin):
        X = np.ascontiguousarray(X_cts, np.uint64)
        nc, level = X.shape[0], X.shape[2] - 1
        X_mu = np.zeros((nc, 2, level, self.N), np.uint64)
        var = np.zeros((2, level - 2, self.N), np.uint64)
        keys = [np.ascontiguousarray(k, np.uint64) for k in gks]
        arr = (_u64p * max(1, len(keys)))(*[_p(k, _u64p) for k in keys])
        relin = np.ascontiguousarray(relin, np.uint64)
        rc = lib().orc_layernorm_head(self._pp, _p(X, _u64p), nc, level, L, D, arr, _p(relin, _u64p),
                                      _p(X_mu, _u64p), _p(var, _u64p))
        if rc:
            raise ValueError(f"layernorm_head failed {rc}")
        return X_mu, var

    # -- local parts of the conversions (Alg. 1 steps 3-4, Alg. 2, App. C.3) --
    def r2f_local(self, party, M, level):
        M = np.ascontiguousarray(M, np.uint64).reshape(-1, 2)
        out = np.zeros((level + 1, len(M)), np.uint64)
        lib().orc_r2f_local(self._pp, party, len(M), _p(M, _u64p), level, _p(out, _u64p))
        return out

    def c2m_local(self, party, t, wsh, scale, l=43, sf=13):
        t = np.ascontiguousarray(t, np.uint64)
        wsh = np.ascontiguousarray(wsh, np.uint64)
        out = np.zeros(self.N // 2, np.uint64)
        rc = lib().orc_c2m_local(self._pp, party, _p(t, _u64p), _p(wsh, _u64p), ctypes.c_double(scale), l, sf,
                                 _p(out, _u64p))
        if rc:
            raise ValueError(f"c2m_local failed {rc}")
        return out

    def m2c_local(self, party, x, wsh, level, scale, l=43, sf=13):
        x = np.ascontiguousarray(x, np.uint64)
        wsh = np.ascontiguousarray(wsh, np.uint64)
        out = np.zeros((level + 1, self.N), np.uint64)
        rc = lib().orc_m2c_local(self._pp, party, _p(x, _u64p), _p(wsh, _u64p), len(x), level,
                                 ctypes.c_double(scale), l, sf, _p(out, _u64p))
        if rc:
            raise ValueError(f"m2c_local failed {rc}")
        return out

    def he2mpc(self, ct, seed, nonce):
        ct = np.ascontiguousarray(ct, np.uint64)
        masked = np.zeros((2, 1, self.N), np.uint64)
        share = np.zeros(self.N, np.uint64)
        lib().orc_he2mpc(self._pp, _p(ct, _u64p), ct.shape[1] - 1, ctypes.c_uint64(seed), nonce,
                         _p(masked, _u64p), _p(share, _u64p))
        return masked, share
