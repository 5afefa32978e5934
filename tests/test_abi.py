"""The C ABI without a GPU: the library loads, exports every entry point
include/blb.h declares, selects the same primes as the oracle (host logic),
and reports a clean error instead of computing when no device is present."""
import ctypes
import os
import re

import pytest

import oracle
from paper_2508_19525_b300 import blb, build
from paper_2508_19525_b300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def read(*parts):
    with open(os.path.join(ROOT, *parts)) as f:
        return f.read()


def declared():
    src = read("include", "blb.h")
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = set(re.findall(r"\b(blb_[a-z0-9_]+)\s*\(", src))
    return names - {"blb_alloc_fn", "blb_free_fn"}


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    L = blb.lib()
    names = declared()
    assert len(names) >= 30
    for n in sorted(names):
        assert hasattr(L, n), n
    assert set(blb.SIGNATURES) == names


def test_binding_has_no_oracle_dependency():
    src = read("paper_2508_19525_b300", "blb.py")
    assert "oracle" not in re.sub(r'""".*?"""', "", src, flags=re.S)
    for f in os.listdir(os.path.join(ROOT, "paper_2508_19525_b300", "csrc")):
        assert "oracle" not in read("paper_2508_19525_b300", "csrc", f)


@pytest.mark.parametrize("prm", [wl.TINY, wl.SMALL, wl.BERT_CP, wl.BERT_CC])
def test_host_prime_selection_matches_oracle(prm):
    assert blb.params_primes(prm.logN, prm.q_bits, prm.p_bits, prm.dnum) == \
        oracle.Oracle(prm.logN, prm.q_bits, prm.p_bits, prm.dnum).primes


@pytest.mark.parametrize("bad", [
    dict(logN=9, q=(50,), p=(60,), dnum=1),         # N too small
    dict(logN=12, q=(50, 40, 40), p=(60,), dnum=1),  # nP < ceil(nQ/dnum)
    dict(logN=12, q=(12,), p=(60,), dnum=1),        # prime too small for 2N
    dict(logN=12, q=(63,), p=(60,), dnum=1),        # prime too large
])
def test_host_parameter_validation(bad):
    with pytest.raises(blb.BlbError):
        blb.params_primes(bad["logN"], bad["q"], bad["p"], bad["dnum"])


def test_context_without_device_fails_cleanly():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    p, keep = blb._params(12, (50, 40, 40), (60,), 3, 2.0 ** 40)
    h = ctypes.c_void_p()
    rc = blb.lib().blb_ctx_create(ctypes.byref(p), None, ctypes.byref(h))
    assert rc == blb.ERR_CUDA and not h.value
    assert blb.last_error()


def test_peaks_library_exports_its_declared_symbols():
    """The benchmark's integer-rate microbenchmarks live in a library of their
    own (include/blb_peaks.h, libblb_peaks.so), not in libblb.so."""
    src = re.sub(r"/\*.*?\*/", "", read("include", "blb_peaks.h"), flags=re.S)
    names = set(re.findall(r"\b(blb_[a-z0-9_]+)\s*\(", src))
    assert names == {"blb_peaks_int_rates", "blb_peaks_reduce_rate"}
    L = ctypes.CDLL(build.build_peaks())
    for n in names:
        assert hasattr(L, n)
        assert not hasattr(blb.lib(), n)
