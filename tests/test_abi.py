"""The C ABI: the library builds, loads and exports every declared entry point.

CPU only: no compute call is made (there may be no GPU here).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cup_gb300.h")


def _declared():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(cup_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib_path():
    from paper_1112_5717_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("cup_factor", "cup_rank_profile", "cup_rref", "cup_det", "cup_inverse",
                 "cup_solve", "cup_mm_sub", "cup_trsm_ruu", "cup_laswp_cols", "cup_create",
                 "cup_destroy"):
        assert must in names


def test_library_exports_every_declared_symbol(lib_path):
    lib = ctypes.CDLL(lib_path)
    for name in _declared():
        assert hasattr(lib, name), name


def test_binding_covers_the_header(lib_path):
    import paper_1112_5717_gb300 as cup
    assert sorted(cup.SIGNATURES) == _declared()
    lib = cup.load()
    for name in cup.SIGNATURES:
        assert getattr(lib, name).argtypes is not None


def test_status_codes_match_header():
    import paper_1112_5717_gb300 as cup
    text = open(HEADER).read()
    for name, val in re.findall(r"(CUP_[A-Z_]+)\s*=\s*(-?\d+)", text):
        if name.startswith(("CUP_OK", "CUP_SINGULAR", "CUP_INCONSISTENT", "CUP_ERR")):
            assert cup.STATUS[int(val)] == name


def test_null_handle_is_rejected(lib_path):
    import paper_1112_5717_gb300 as cup
    lib = cup.load()
    r = ctypes.c_int64(0)
    assert lib.cup_factor(None, None, 0, 0, 1, 7, None, None, ctypes.byref(r), None) == -1
    assert lib.cup_set_option(None, 0, 0) == -1
    assert lib.cup_destroy(None) == -1


def _trial_prime(q: int) -> bool:
    if q < 2:
        return False
    d = 2
    while d * d <= q:
        if q % d == 0:
            return False
        d += 1
    return True


def test_primes_below_against_trial_division(lib_path):
    """Host prime generator of the multi-modular path: the largest primes below a bound."""
    import paper_1112_5717_gb300 as cup
    got = cup.primes_below(1 << 31, 12)
    want, q = [], (1 << 31) - 1
    while len(want) < 12:
        if _trial_prime(q):
            want.append(q)
        q -= 1
    assert got == want
    assert cup.primes_below(100, 1000) == [q for q in range(99, 1, -1) if _trial_prime(q)]
    assert cup.primes_below(2, 5) == []


def test_crt_symmetric_range(lib_path):
    """Host Chinese remaindering (mixed radix): every x in (-M/2, M/2] comes back
    from its residues, including both ends of the range and zero."""
    import random

    import paper_1112_5717_gb300 as cup
    rnd = random.Random(5)
    for K in (1, 2, 7, 40):
        primes = cup.primes_below((1 << 31) - rnd.randrange(1 << 20), K)
        M = 1
        for q in primes:
            M *= q
        cases = [0, 1, -1, (M - 1) // 2, -((M - 1) // 2)] + [rnd.randrange(-(M // 2), M // 2) for _ in range(20)]
        for x in cases:
            assert cup.crt([x % q for q in primes], primes) == x
    small = [5, 7, 11]
    for x in range(-192, 193):                    # M = 385: all of (-M/2, M/2]
        assert cup.crt([x % q for q in small], small) == x


def test_crt_rejects_bad_primes(lib_path):
    import paper_1112_5717_gb300 as cup
    with pytest.raises(cup.CupError) as e:
        cup.crt([1, 2], [65521, 65521])
    assert e.value.status == -1
    with pytest.raises(cup.CupError) as e:
        cup.crt([1, 2], [65521, 65522])
    assert e.value.status == -2
    lib = cup.load()
    r = (ctypes.c_uint32 * 3)(1, 2, 3)
    q = (ctypes.c_uint32 * 3)(*cup.primes_below(1 << 31, 3))
    w = (ctypes.c_uint32 * 1)()
    nw, sg = ctypes.c_int64(0), ctypes.c_int(0)
    assert lib.cup_crt(r, q, 3, w, 1, ctypes.byref(nw), ctypes.byref(sg)) == -8
    assert nw.value >= 2


def test_every_dependent_launch_waits_for_its_predecessor():
    """Kernels launched with programmatic dependent launch may start while the
    previous kernel of their stream is still running; each of them must pass
    pdl_enter() (griddepcontrol.wait) in its body. Checked on the sources."""
    csrc = os.path.join(ROOT, "paper_1112_5717_gb300", "csrc")
    text = "".join(open(os.path.join(csrc, f)).read() for f in sorted(os.listdir(csrc)) if f.endswith(".cu"))
    launched = set(re.findall(r"launch_pdl\((k_\w+|tc::k_\w+|k_\w+<)", text))
    launched = {n.replace("tc::", "").rstrip("<") for n in launched}
    assert len(launched) >= 10
    for name in sorted(launched):
        m = re.search(r"__global__[^;{]*?\b" + name + r"\s*\([^{]*\{", text, flags=re.S)
        assert m, name
        # the kernel's body up to its matching brace
        depth, j = 1, m.end()
        while depth:
            depth += {"{": 1, "}": -1}.get(text[j], 0)
            j += 1
        assert "pdl_enter();" in text[m.end():j], name
