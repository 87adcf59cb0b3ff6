"""CPU oracle for the RNS-CKKS worker arithmetic (Li & Huang, KDD'20, Sec. 3-4).

TEST INFRASTRUCTURE ONLY.  Only the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg import this package.  The product library never
loads it, and the two share no code: this binding only marshals numpy arrays
into ``he_oracle.c``, which computes every residue with exact ``__int128``
arithmetic from the textbook definitions.

Parity status: every function here is pinned by the ``-m "not gpu"`` tests in
``tests/test_oracle_*.py`` against something other than itself (brute force,
closed forms, library routines, big-integer reconstructions, FP64 plaintext
computations).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "he_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

U64P = ctypes.POINTER(ctypes.c_uint64)
I64P = ctypes.POINTER(ctypes.c_int64)
DBLP = ctypes.POINTER(ctypes.c_double)
VP = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile he_oracle.c into liboracle.so (gcc, no FMA contraction so
    that double scale bookkeeping is the same on every host), with OpenMP
    when the compiler has it (results do not depend on the thread count)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp, _SRC]
        if subprocess.call(base[:1] + ["-fopenmp"] + base[1:] + ["-lm"], stderr=subprocess.DEVNULL) != 0:
            subprocess.check_call(base + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def set_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (OpenMP; 1 without it)."""
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            lib.orc_create.restype = VP
            lib.orc_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint64, VP, ctypes.c_int]
            lib.orc_destroy.argtypes = [VP]
            lib.orc_set_threads.argtypes = [ctypes.c_int]
            lib.orc_get_threads.restype = ctypes.c_int
            lib.orc_is_prime.argtypes = [ctypes.c_uint64]
            lib.orc_min_root.restype = ctypes.c_uint64
            lib.orc_min_root.argtypes = [ctypes.c_uint64, ctypes.c_int]
            lib.orc_galois_elt.restype = ctypes.c_uint64
            lib.orc_galois_elt.argtypes = [ctypes.c_int, ctypes.c_int32]
            lib.orc_gen_primes.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, VP,
                                           ctypes.c_int, VP]
            lib.orc_gauss_table.argtypes = [ctypes.c_double, VP]
            lib.orc_sample.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                       ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                       ctypes.c_double, ctypes.c_uint32, VP]
            for name in ("orc_ntt_def", "orc_intt_def"):
                getattr(lib, name).argtypes = [VP, VP, ctypes.c_int, ctypes.c_uint64,
                                               ctypes.c_uint64]
            for name in ("orc_ntt_r2", "orc_intt_r2"):
                getattr(lib, name).argtypes = [VP, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]
            lib.orc_automorph_coef.argtypes = [VP, VP, ctypes.c_int, ctypes.c_uint64,
                                               ctypes.c_uint64]
            lib.orc_philox.argtypes = [VP, VP, VP]
            lib.orc_encode_raw.argtypes = [VP, VP, VP, ctypes.c_int, ctypes.c_double, VP]
            lib.orc_encode.argtypes = [VP, VP, VP, ctypes.c_int, ctypes.c_double, VP]
            lib.orc_decode.argtypes = [VP, VP, ctypes.c_double, VP, VP]
            lib.orc_encrypt.argtypes = [VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_uint32, VP]
            lib.orc_decrypt.argtypes = [VP, VP, ctypes.c_int, VP, VP, ctypes.c_int, VP]
            for name in ("orc_add", "orc_sub"):
                getattr(lib, name).argtypes = [VP, VP, VP, ctypes.c_int, VP]
            lib.orc_drop.argtypes = [VP, VP, ctypes.c_int, ctypes.c_int, VP]
            lib.orc_mul_int.argtypes = [VP, VP, ctypes.c_int, ctypes.c_int64, VP]
            lib.orc_add_int.argtypes = [VP, VP, ctypes.c_int, ctypes.c_int64, VP]
            lib.orc_mul_plain.argtypes = [VP, VP, ctypes.c_int, VP, VP]
            lib.orc_tensor.argtypes = [VP, VP, VP, ctypes.c_int, VP]
            lib.orc_modup_coef.argtypes = [VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_int, VP]
            lib.orc_moddown_conv.argtypes = [VP, VP, ctypes.c_int, VP]
            lib.orc_keyswitch.argtypes = [VP, VP, ctypes.c_int, ctypes.c_int, VP, VP]
            lib.orc_moddown.argtypes = [VP, VP, ctypes.c_int, VP, VP]
            lib.orc_moddown_rescale.argtypes = [VP, VP, VP, ctypes.c_int, VP]
            lib.orc_rescale.argtypes = [VP, VP, ctypes.c_int, VP]
            lib.orc_mul_relin_rescale.argtypes = [VP, VP, VP, ctypes.c_int, VP]
            lib.orc_mul_relin.argtypes = [VP, VP, VP, ctypes.c_int, VP]
            lib.orc_rotate.argtypes = [VP, VP, ctypes.c_int, ctypes.c_int32, VP]
            lib.orc_rotate_sum.argtypes = [VP, VP, ctypes.c_int, VP, ctypes.c_int, VP]
            lib.orc_automorph.argtypes = [VP, VP, VP, ctypes.c_int, ctypes.c_uint64]
            lib.orc_get_primes.argtypes = [VP, VP]
            lib.orc_get_roots.argtypes = [VP, VP]
            lib.orc_get_secret.argtypes = [VP, VP]
            lib.orc_get_beta.argtypes = [VP]
            lib.orc_get_key.argtypes = [VP, ctypes.c_int, VP]
            lib.orc_lr_mask.argtypes = [VP, ctypes.c_int, ctypes.c_double, VP]
            lib.orc_lr_inference.argtypes = [
                VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_double, VP, ctypes.c_int, ctypes.c_double,
                VP, ctypes.c_double, ctypes.c_int, VP, VP]
            lib.orc_lr_gradient_step.argtypes = [
                VP, VP, ctypes.c_int, ctypes.c_int, ctypes.c_double, VP, ctypes.c_int,
                ctypes.c_double, VP, ctypes.c_double, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                VP, VP, VP]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def _u64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint64)


# --------------------------------------------------------------------------
# Stand-alone primitives
# --------------------------------------------------------------------------

def is_prime(n: int) -> bool:
    return bool(_load().orc_is_prime(n))


def gen_primes(bits: int, log_n: int, count: int, exclude=()) -> list[int]:
    out = np.zeros(count, dtype=np.uint64)
    ex = _u64(list(exclude) or [0])
    got = _load().orc_gen_primes(bits, log_n, count, _p(ex), len(exclude), _p(out))
    return [int(x) for x in out[:got]]


def min_root(q: int, log_n: int) -> int:
    return int(_load().orc_min_root(q, log_n))


def galois_elt(log_n: int, r: int) -> int:
    return int(_load().orc_galois_elt(log_n, r))


def gauss_table(sigma: float) -> np.ndarray:
    t = np.zeros(256, dtype=np.uint64)
    k = _load().orc_gauss_table(sigma, _p(t))
    return t[:k].copy()


def philox(ctr, key) -> np.ndarray:
    c = np.asarray(ctr, dtype=np.uint32)
    k = np.asarray(key, dtype=np.uint32)
    o = np.zeros(4, dtype=np.uint32)
    _load().orc_philox(_p(c), _p(k), _p(o))
    return o


def sample(seed: int, kind: str, sid: int, dom: int, count: int, limb: int = 0, q: int = 1,
           sigma: float = 3.2) -> np.ndarray:
    kinds = {"ternary": 0, "gauss": 1, "uniform": 2}
    out = np.zeros(count, dtype=np.int64)
    _load().orc_sample(seed, kinds[kind], sid, dom, limb, q, sigma, count, _p(out))
    return out


def ntt_def(a, log_n: int, q: int, psi: int) -> np.ndarray:
    a = _u64(a)
    out = np.zeros_like(a)
    _load().orc_ntt_def(_p(a), _p(out), log_n, q, psi)
    return out


def intt_def(a, log_n: int, q: int, psi: int) -> np.ndarray:
    a = _u64(a)
    out = np.zeros_like(a)
    _load().orc_intt_def(_p(a), _p(out), log_n, q, psi)
    return out


def ntt_r2(a, log_n: int, q: int, psi: int) -> np.ndarray:
    a = _u64(a).copy()
    _load().orc_ntt_r2(_p(a), log_n, q, psi)
    return a


def intt_r2(a, log_n: int, q: int, psi: int) -> np.ndarray:
    a = _u64(a).copy()
    _load().orc_intt_r2(_p(a), log_n, q, psi)
    return a


def automorph_coef(a, log_n: int, q: int, k: int) -> np.ndarray:
    a = _u64(a)
    out = np.zeros_like(a)
    _load().orc_automorph_coef(_p(a), _p(out), log_n, q, k)
    return out


# --------------------------------------------------------------------------
# Context
# --------------------------------------------------------------------------

def fit_poly(x, y, degree: int) -> np.ndarray:
    """Least-squares polynomial fit (Sec. 3, Eq. 3), by its definition: the
    coefficients c minimising ||V c - y||_2 for the Vandermonde matrix
    V[i, k] = x_i^k, from numpy's least-squares solver (SVD based)."""
    x = np.asarray(x, dtype=np.float64)
    V = np.vander(x, degree + 1, increasing=True)
    c, *_ = np.linalg.lstsq(V, np.asarray(y, dtype=np.float64), rcond=None)
    return c


class Ciphertext:
    """Residues [2][level][N] (uint64, evaluation form), level and scale."""

    def __init__(self, data: np.ndarray, level: int, scale: float):
        self.data = data
        self.level = level
        self.scale = scale


class Oracle:
    """Keys and parameters generated from a seed, as in the product's
    ``he_ctx_create``; all methods return fresh numpy arrays."""

    def __init__(self, log_n: int, n_limbs: int, limb_bits: int, n_special: int,
                 special_bits: int, scale: float, sigma: float = 3.2, seed: int = 0,
                 rot_steps=()):
        lib = _load()
        rots = np.asarray(list(rot_steps) or [0], dtype=np.int32)
        self._lib = lib
        self.ptr = lib.orc_create(log_n, n_limbs, limb_bits, n_special, special_bits,
                                  float(scale), float(sigma), seed, _p(rots), len(rot_steps))
        if not self.ptr:
            raise ValueError("oracle: bad parameters")
        self.log_n, self.n, self.L, self.alpha = log_n, 1 << log_n, n_limbs, n_special
        self.scale, self.sigma, self.seed = float(scale), float(sigma), seed
        self.rot_steps = list(rot_steps)
        self.np_ = n_limbs + n_special
        pr = np.zeros(self.np_, dtype=np.uint64)
        lib.orc_get_primes(self.ptr, _p(pr))
        self.primes = [int(x) for x in pr]
        rt = np.zeros(self.np_, dtype=np.uint64)
        lib.orc_get_roots(self.ptr, _p(rt))
        self.roots = [int(x) for x in rt]
        self.beta = lib.orc_get_beta(self.ptr)
        # Galois keys are stored in creation order, skipping duplicates/identity.
        self.gal_order = []
        for r in rot_steps:
            k = galois_elt(log_n, r)
            if k != 1 and k not in self.gal_order:
                self.gal_order.append(k)

    def __del__(self):
        if getattr(self, "ptr", None):
            self._lib.orc_destroy(self.ptr)
            self.ptr = None

    # -- keys --------------------------------------------------------------
    def secret(self) -> np.ndarray:
        s = np.zeros(self.n, dtype=np.int8)
        self._lib.orc_get_secret(self.ptr, _p(s))
        return s

    def key(self, which: int) -> np.ndarray:
        if which == 0:
            out = np.zeros((2, self.L, self.n), dtype=np.uint64)
        else:
            out = np.zeros((self.beta, 2, self.np_, self.n), dtype=np.uint64)
        rc = self._lib.orc_get_key(self.ptr, which, _p(out))
        if rc:
            raise KeyError(which)
        return out

    # -- encode/decode -------------------------------------------------------
    def encode_raw(self, re, im=None, scale=None) -> np.ndarray:
        re = np.ascontiguousarray(re, dtype=np.float64)
        imv = None if im is None else np.ascontiguousarray(im, dtype=np.float64)
        out = np.zeros(self.n, dtype=np.float64)
        self._lib.orc_encode_raw(self.ptr, _p(re), _p(imv) if imv is not None else None,
                                 len(re), float(scale or self.scale), _p(out))
        return out

    def encode(self, re, im=None, scale=None) -> np.ndarray:
        re = np.ascontiguousarray(re, dtype=np.float64)
        imv = None if im is None else np.ascontiguousarray(im, dtype=np.float64)
        out = np.zeros(self.n, dtype=np.int64)
        rc = self._lib.orc_encode(self.ptr, _p(re), _p(imv) if imv is not None else None,
                                  len(re), float(scale or self.scale), _p(out))
        if rc:
            raise OverflowError("encode: coefficient beyond int64")
        return out

    def decode(self, mcoef, scale: float):
        m = np.ascontiguousarray(mcoef, dtype=np.float64)
        re = np.zeros(self.n // 2, dtype=np.float64)
        im = np.zeros(self.n // 2, dtype=np.float64)
        self._lib.orc_decode(self.ptr, _p(m), float(scale), _p(re), _p(im))
        return re, im

    # -- encrypt/decrypt ----------------------------------------------------
    def encrypt(self, m, level: int, use_sk: bool = False, cid: int = 0,
                scale: float | None = None) -> Ciphertext:
        m = np.ascontiguousarray(m, dtype=np.int64)
        out = np.zeros((2, level, self.n), dtype=np.uint64)
        rc = self._lib.orc_encrypt(self.ptr, _p(m), level, int(use_sk), cid, _p(out))
        if rc:
            raise ValueError("encrypt: bad level")
        return Ciphertext(out, level, float(scale or self.scale))

    def decrypt_coeffs(self, ct: Ciphertext, exact: bool = False):
        """Centered coefficients of c0 + c1 s; as doubles, or (exact=True) as
        Python integers."""
        d = _u64(ct.data)
        out = np.zeros(self.n, dtype=np.float64)
        if not exact:
            self._lib.orc_decrypt(self.ptr, _p(d), ct.level, _p(out), None, 0, None)
            return out
        nw = 32
        words = np.zeros((self.n, nw), dtype=np.uint64)
        signs = np.zeros(self.n, dtype=np.int8)
        self._lib.orc_decrypt(self.ptr, _p(d), ct.level, _p(out), _p(words), nw, _p(signs))
        vals = []
        for i in range(self.n):
            v = 0
            for k in range(nw - 1, -1, -1):
                v = (v << 64) | int(words[i, k])
            vals.append(-v if signs[i] else v)
        return vals

    def decrypt(self, ct: Ciphertext):
        """Slots (real parts, imaginary parts) of a ciphertext."""
        m = self.decrypt_coeffs(ct)
        return self.decode(m, ct.scale)

    # -- ops -----------------------------------------------------------------
    def _new(self, level, parts=2):
        return np.zeros((parts, level, self.n), dtype=np.uint64)

    def add(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        out = self._new(a.level)
        self._lib.orc_add(self.ptr, _p(_u64(a.data)), _p(_u64(b.data)), a.level, _p(out))
        return Ciphertext(out, a.level, a.scale)

    def sub(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        out = self._new(a.level)
        self._lib.orc_sub(self.ptr, _p(_u64(a.data)), _p(_u64(b.data)), a.level, _p(out))
        return Ciphertext(out, a.level, a.scale)

    def drop(self, a: Ciphertext, to: int) -> Ciphertext:
        out = self._new(to)
        self._lib.orc_drop(self.ptr, _p(_u64(a.data)), a.level, to, _p(out))
        return Ciphertext(out, to, a.scale)

    def mul_int(self, a: Ciphertext, k: int, scale_k: float = 1.0) -> Ciphertext:
        out = self._new(a.level)
        self._lib.orc_mul_int(self.ptr, _p(_u64(a.data)), a.level, int(k), _p(out))
        return Ciphertext(out, a.level, a.scale * scale_k)

    def add_int(self, a: Ciphertext, k: int) -> Ciphertext:
        out = self._new(a.level)
        self._lib.orc_add_int(self.ptr, _p(_u64(a.data)), a.level, int(k), _p(out))
        return Ciphertext(out, a.level, a.scale)

    def mul_plain(self, a: Ciphertext, m, scale_m: float) -> Ciphertext:
        m = np.ascontiguousarray(m, dtype=np.int64)
        out = self._new(a.level)
        self._lib.orc_mul_plain(self.ptr, _p(_u64(a.data)), a.level, _p(m), _p(out))
        return Ciphertext(out, a.level, a.scale * scale_m)

    def tensor(self, a: Ciphertext, b: Ciphertext) -> np.ndarray:
        out = self._new(a.level, 3)
        self._lib.orc_tensor(self.ptr, _p(_u64(a.data)), _p(_u64(b.data)), a.level, _p(out))
        return out

    def modup_coef(self, xcoef, level: int, digit: int, prime_index: int) -> np.ndarray:
        x = _u64(xcoef)
        out = np.zeros(self.n, dtype=np.uint64)
        self._lib.orc_modup_coef(self.ptr, _p(x), level, digit, prime_index, _p(out))
        return out

    def moddown_conv(self, ycoefP, t: int) -> np.ndarray:
        y = _u64(ycoefP)
        out = np.zeros(self.n, dtype=np.uint64)
        self._lib.orc_moddown_conv(self.ptr, _p(y), t, _p(out))
        return out

    def keyswitch(self, d, level: int, key_id: int = -1):
        d = _u64(d)
        k0 = np.zeros((level, self.n), dtype=np.uint64)
        k1 = np.zeros((level, self.n), dtype=np.uint64)
        rc = self._lib.orc_keyswitch(self.ptr, _p(d), level, key_id, _p(k0), _p(k1))
        if rc:
            raise KeyError(key_id)
        return k0, k1

    def moddown(self, acc, level: int):
        """round(acc / P) of an accumulator [2][level + alpha][N] (evaluation
        form): the key switch's last step (orc_moddown)."""
        a = _u64(acc)
        k0 = np.zeros((level, self.n), dtype=np.uint64)
        k1 = np.zeros((level, self.n), dtype=np.uint64)
        if self._lib.orc_moddown(self.ptr, _p(a), level, _p(k0), _p(k1)):
            raise ValueError("moddown: level")
        return k0, k1

    def moddown_rescale(self, acc, d01, level: int) -> np.ndarray:
        """round((P d01 + acc) / (P q_{level-1})), the multiplication's merged
        ModDown and rescale (orc_moddown_rescale): [2][level-1][N]."""
        a, d = _u64(acc), _u64(d01)
        out = np.zeros((2, level - 1, self.n), dtype=np.uint64)
        if self._lib.orc_moddown_rescale(self.ptr, _p(a), _p(d), level, _p(out)):
            raise ValueError("moddown_rescale: level")
        return out

    def rescale(self, a: Ciphertext) -> Ciphertext:
        out = self._new(a.level - 1)
        rc = self._lib.orc_rescale(self.ptr, _p(_u64(a.data)), a.level, _p(out))
        if rc:
            raise ValueError("rescale: level")
        return Ciphertext(out, a.level - 1, a.scale / self.primes[a.level - 1])

    def mul_relin_rescale(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        out = self._new(a.level - 1)
        rc = self._lib.orc_mul_relin_rescale(self.ptr, _p(_u64(a.data)), _p(_u64(b.data)),
                                             a.level, _p(out))
        if rc:
            raise ValueError("mul_relin_rescale: level")
        return Ciphertext(out, a.level - 1, a.scale * b.scale / self.primes[a.level - 1])

    def mul_relin(self, a: Ciphertext, b: Ciphertext) -> Ciphertext:
        out = self._new(a.level)
        self._lib.orc_mul_relin(self.ptr, _p(_u64(a.data)), _p(_u64(b.data)), a.level, _p(out))
        return Ciphertext(out, a.level, a.scale * b.scale)

    def rotate(self, a: Ciphertext, r: int) -> Ciphertext:
        out = self._new(a.level)
        rc = self._lib.orc_rotate(self.ptr, _p(_u64(a.data)), a.level, r, _p(out))
        if rc:
            raise KeyError(f"no Galois key for rotation {r}")
        return Ciphertext(out, a.level, a.scale)

    def rotate_sum(self, a: Ciphertext, steps) -> Ciphertext:
        """a + sum_s rot(a, s) with one shared decomposition of a's second part
        (orc_rotate_sum)."""
        st = np.ascontiguousarray(steps, dtype=np.int32)
        out = self._new(a.level)
        rc = self._lib.orc_rotate_sum(self.ptr, _p(_u64(a.data)), a.level, _p(st), len(st), _p(out))
        if rc:
            raise KeyError(f"rotate_sum {list(steps)} failed ({rc})")
        return Ciphertext(out, a.level, a.scale)

    def automorph(self, polys, nlimbs: int, k: int) -> np.ndarray:
        a = _u64(polys)
        out = np.zeros_like(a)
        self._lib.orc_automorph(self.ptr, _p(a), _p(out), nlimbs, k)
        return out

    def lr_mask(self, g: int, mask_scale: float) -> np.ndarray:
        out = np.zeros(self.n, dtype=np.int64)
        self._lib.orc_lr_mask(self.ptr, g, float(mask_scale), _p(out))
        return out

    def lr_gradient_step(self, Z: list, W: Ciphertext, coeffs, lr: float, g: int,
                         mask_scale: float, l2: float = 0.0) -> Ciphertext:
        """w' = w + lr (sum_i p(y_i w.x_i) y_i x_i - l2 w) (orc_lr_gradient_step)."""
        arrs = [_u64(z.data) for z in Z]
        ptrs = np.array([a.ctypes.data for a in arrs], dtype=np.uint64)
        co = np.ascontiguousarray(coeffs, dtype=np.float64)
        out = self._new(W.level - 5)
        lvl = ctypes.c_int(0)
        sc = ctypes.c_double(0.0)
        rc = self._lib.orc_lr_gradient_step(
            self.ptr, _p(ptrs), len(Z), Z[0].level, float(Z[0].scale), _p(_u64(W.data)),
            W.level, float(W.scale), _p(co), float(lr), g, float(mask_scale), float(l2), _p(out),
            ctypes.byref(lvl), ctypes.byref(sc))
        if rc:
            raise ValueError(f"lr_gradient_step failed ({rc})")
        return Ciphertext(out, lvl.value, sc.value)

    def lr_inference(self, Z: list, W: Ciphertext, coeffs, lr: float, g: int) -> list:
        """S_k = p(M_k) for each data ciphertext (level W.level - 3)."""
        arrs = [_u64(z.data) for z in Z]
        ptrs = np.array([a.ctypes.data for a in arrs], dtype=np.uint64)
        co = np.ascontiguousarray(coeffs, dtype=np.float64)
        lv = W.level - 3
        out = np.zeros((len(Z), 2, lv, self.n), dtype=np.uint64)
        sc = ctypes.c_double(0.0)
        rc = self._lib.orc_lr_inference(self.ptr, _p(ptrs), len(Z), Z[0].level, float(Z[0].scale),
                                         _p(_u64(W.data)), W.level, float(W.scale), _p(co), float(lr), g,
                                         _p(out), ctypes.byref(sc))
        if rc:
            raise ValueError(f"lr_inference failed ({rc})")
        return [Ciphertext(out[k], lv, sc.value) for k in range(len(Z))]
