"""Seeded synthetic inputs with the shapes and value distributions of the
paper's workloads (BERT-base / BERT-large / GPT2-base shaped operands, Sec. 7).

This module only draws numbers: it holds none of the method's arithmetic, and
both the CUDA path's tests and the CPU oracle consume the same arrays.  The
paper evaluates on GLUE (Sec. 7.1); those data and trained weights are not
used -- matrices of the same shapes stand in for them.
"""
from dataclasses import dataclass, field
from typing import List

import numpy as np


@dataclass(frozen=True)
class HEParams:
    logN: int
    q_bits: tuple
    p_bits: tuple
    dnum: int
    scale: float = float(2 ** 40)

    @property
    def N(self):
        return 1 << self.logN

    @property
    def slots(self):
        return self.N // 2


# Parameter sets.  Bit widths: a 60-bit (or 50-bit) base prime q_0, 40-bit
# primes for every rescale at scale 2^40, 60-bit special primes for key
# switching (alpha = ceil(nQ/dnum) of them).
TINY = HEParams(12, (50, 40, 40), (60,), 3)                       # N=2^12, 3 primes
BERT_CP = HEParams(15, (60,) + (40,) * 7, (60,) * 3, 3)           # N=2^15, 8 primes, dnum 3
BERT_CC = HEParams(16, (60,) + (40,) * 11, (60,) * 3, 4)          # N=2^16, 12 primes, dnum 4
# small parameter sets for fast parity runs (several limbs, several digits)
SMALL = HEParams(12, (60, 40, 40, 40, 40), (60, 60), 3)           # 5 primes, dnum 3 (alpha 2)
MICRO = HEParams(5, (50, 40, 40), (60,), 3)                       # N=32, schoolbook-checkable


def uniform(shape, seed, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)


def cp_operands(m, d, d_out, seed):
    """X (m x d) and W (d x d_out), both U[-1, 1] (FP64)."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, size=(m, d))
    W = rng.uniform(-1.0, 1.0, size=(d, d_out))
    return X, W


def bert_base_cp(seed=0):
    """X 128x768, W_QKV 768x2304, W_O 768x768, U[-1, 1]."""
    rng = np.random.default_rng(seed)
    X = rng.uniform(-1.0, 1.0, size=(128, 768))
    W_qkv = rng.uniform(-1.0, 1.0, size=(768, 2304))
    W_o = rng.uniform(-1.0, 1.0, size=(768, 768))
    return X, W_qkv, W_o


def attention_operands(L, H, Dh, seed=0):
    """Q, K, V ~ N(0, 0.5) clipped to [-1, 1] (0.5 read as the standard
    deviation); P rows Dirichlet(1) (softmax-like, rows sum to 1)."""
    rng = np.random.default_rng(seed)
    Q = np.clip(rng.normal(0.0, 0.5, size=(H, L, Dh)), -1.0, 1.0)
    K = np.clip(rng.normal(0.0, 0.5, size=(H, L, Dh)), -1.0, 1.0)
    V = np.clip(rng.normal(0.0, 0.5, size=(H, L, Dh)), -1.0, 1.0)
    P = rng.dirichlet(np.ones(L), size=(H, L))
    return Q, K, V, P


def slot_vector(n, seed, lo=-1.0, hi=1.0):
    return np.random.default_rng(seed).uniform(lo, hi, size=n)


def random_residues(primes, N, seed, polys=1):
    """Uniform residues: array (polys, len(primes), N) with limb i mod primes[i]."""
    rng = np.random.default_rng(seed)
    out = np.zeros((polys, len(primes), N), np.uint64)
    for p in range(polys):
        for i, q in enumerate(primes):
            out[p, i] = rng.integers(0, q, size=N, dtype=np.uint64)
    return out
