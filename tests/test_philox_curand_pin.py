"""Known-answer pin of the oracle's Philox4x32-10 against an independent implementation.

cuRAND's host-side generator CURAND_RNG_PSEUDO_PHILOX4_32_10 (run here, on the CPU,
through its public C API) is an implementation of the same generator of Salmon et
al. (SC'11) that the Gaussian test matrix of Sec. 3.3 is drawn from.  With the
default ordering its output word j is word j % 4 of Philox4x32-10 on the counter
(r, 0, t, 0) with the key (seed low, seed high), where b = j // 4, t = b % 65536
and r = b // 65536: 65,536 subsequences t (counter words 2-3) advanced together
round by round r (counter words 0-1).  That is the same counter and key layout
the oracle's Gaussian transform uses (variate pair index in words 0-1, stream in
words 2-3, seed as the key), so word-for-word agreement pins the multipliers, the
Weyl constants, the round function and the counter/key placement.  A planted
one-bit change to any of the four constants in a copy of the oracle must fail the
comparison.
"""
import ctypes as C
import ctypes.util
import glob
import os
import re
import subprocess

import numpy as np
import pytest

import oracle

PHILOX = 161          # CURAND_RNG_PSEUDO_PHILOX4_32_10 (curand.h)
THREADS = 65536       # subsequences of the host generator's default ordering


def _curand():
    cands = []
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d:
            cands += sorted(glob.glob(os.path.join(d, "lib64", "libcurand.so*")))
            cands += sorted(glob.glob(os.path.join(d, "targets", "*", "lib", "libcurand.so*")))
    lib = ctypes.util.find_library("curand")
    if lib:
        cands.append(lib)
    for c in cands:
        try:
            return C.CDLL(c)
        except OSError:
            continue
    pytest.skip("libcurand not found")


def _curand_words(seed: int, n: int) -> np.ndarray:
    lib = _curand()
    gen = C.c_void_p()
    assert lib.curandCreateGeneratorHost(C.byref(gen), PHILOX) == 0
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, C.c_ulonglong(seed)) == 0
        out = np.zeros(n, dtype=np.uint32)
        assert lib.curandGenerate(gen, out.ctypes.data_as(C.c_void_p), C.c_size_t(n)) == 0
    finally:
        lib.curandDestroyGenerator(gen)
    return out


def _blocks(nblocks, rng):
    picks = {0, 1, THREADS - 1, THREADS, THREADS + 1, nblocks - 1}
    picks |= set(int(x) for x in rng.integers(0, nblocks, 600))
    return sorted(picks)


def _expected(philox, seed, b):
    r, t = divmod(b, THREADS)
    return philox([r, 0, t, 0], [seed & 0xFFFFFFFF, seed >> 32])


@pytest.mark.parametrize("seed", [0, 1234, 0x9E3779B97F4A7C15, (1 << 64) - 1])
def test_oracle_philox_matches_curand_word_for_word(seed):
    nblocks = 3 * THREADS  # three rounds of every subsequence
    words = _curand_words(seed, 4 * nblocks)
    rng = np.random.default_rng(seed & 0xFFFF)
    for b in _blocks(nblocks, rng):
        assert _expected(oracle.philox4x32, seed, b) == [int(x) for x in words[4 * b:4 * b + 4]], b


def test_gaussian_counter_layout_matches_curand_subsequences():
    # the oracle's Gaussian variate pair p of stream s draws Philox on counter
    # (p, 0, s, 0): the same words cuRAND emits for subsequence s in round p
    seed = 2024
    words = _curand_words(seed, 4 * 2 * THREADS)
    for s, p in [(0, 0), (7, 1), (65535, 1), (300, 0)]:
        b = p * THREADS + s
        w = [int(x) for x in words[4 * b:4 * b + 4]]
        u1 = 1.0 - (((w[0] >> 5) << 26) | (w[1] >> 6)) * 2.0 ** -53
        u2 = (((w[2] >> 5) << 26) | (w[3] >> 6)) * 2.0 ** -53
        r = np.sqrt(-2.0 * np.log(u1))
        g = oracle.gaussian(seed, s, 2, first=2 * p)
        assert abs(g[0] - r * np.cos(2 * np.pi * u2)) <= 1e-12 * max(1.0, r)
        assert abs(g[1] - r * np.sin(2 * np.pi * u2)) <= 1e-12 * max(1.0, r)


def _mutant_philox(tmp_path, name: str, bit: int):
    """A copy of the oracle's source with one bit of one Philox constant flipped."""
    src = open(os.path.join(os.path.dirname(oracle.__file__), "oracle.c")).read()
    m = re.search(r"(%s = )0x([0-9A-Fa-f]+)u" % name, src)
    assert m, name
    val = int(m.group(2), 16) ^ (1 << bit)
    mutated = src[:m.start()] + f"{m.group(1)}0x{val:08X}u" + src[m.end():]
    c_path = tmp_path / f"mut_{name}_{bit}.c"
    so_path = tmp_path / f"mut_{name}_{bit}.so"
    c_path.write_text(mutated)
    subprocess.run([os.environ.get("CC", "gcc"), "-O1", "-fPIC", "-shared", "-std=c11",
                    "-ffp-contract=off", "-o", str(so_path), str(c_path), "-lm"], check=True)
    lib = C.CDLL(str(so_path))
    u32p = C.POINTER(C.c_uint32)
    lib.orc_philox4x32.argtypes = [u32p, u32p, C.c_int, u32p]
    lib.orc_philox4x32.restype = None

    def philox(ctr, key):
        c = (C.c_uint32 * 4)(*ctr)
        k = (C.c_uint32 * 2)(*key)
        o = (C.c_uint32 * 4)()
        lib.orc_philox4x32(c, k, 10, o)
        return [int(x) for x in o]

    return philox


@pytest.mark.parametrize("name,bit", [("PH32_M0", 0), ("PH32_M1", 17), ("PH32_W0", 31),
                                      ("PH32_W1", 3)])
def test_planted_constant_mistake_is_caught(tmp_path, name, bit):
    seed = 1234
    words = _curand_words(seed, 4 * 2 * THREADS)
    philox = _mutant_philox(tmp_path, name, bit)
    blocks = [0, 1, 5, THREADS - 1, THREADS, THREADS + 7]
    mismatches = sum(_expected(philox, seed, b) != [int(x) for x in words[4 * b:4 * b + 4]]
                     for b in blocks)
    assert mismatches == len(blocks)
