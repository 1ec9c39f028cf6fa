"""Pins of the oracle's counter-based generator (Philox4x32-10, Salmon et al.
SC'11) and of the uniform conversion, against an independent implementation:
cuRAND's host-side Philox4_32_10 generator, which runs on the CPU."""
import ctypes
import os

import numpy as np
import pytest

import oracle as O
from paper_2312_16981_gb300 import inputs as I

CURAND_RNG_PSEUDO_PHILOX4_32_10 = 161


def _curand():
    cands = [os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "lib64", "libcurand.so"),
             "libcurand.so", "libcurand.so.10"]
    for c in cands:
        try:
            return ctypes.CDLL(c)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def _curand_words(seed: int, n_words: int) -> np.ndarray:
    L = _curand()
    gen = ctypes.c_void_p()
    assert L.curandCreateGeneratorHost(ctypes.byref(gen), CURAND_RNG_PSEUDO_PHILOX4_32_10) == 0
    try:
        assert L.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        out = np.zeros(n_words, dtype=np.uint32)
        assert L.curandGenerate(gen, out.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(n_words)) == 0
    finally:
        L.curandDestroyGenerator(gen)
    return out


@pytest.mark.parametrize("seed", [0, 1, 0x123456789ABCDEF, 0xFFFFFFFF00000001])
def test_philox_matches_curand_host_generator(seed):
    # cuRAND's host Philox emits block b of counter (b // 65536, 0, b % 65536, 0)
    # under key (seed_lo, seed_hi); we check blocks from both counter lanes.
    nblk = 65536 + 64
    words = _curand_words(seed, 4 * nblk).reshape(nblk, 4)
    key = (seed & 0xFFFFFFFF, seed >> 32)
    blocks = list(range(0, 65536, 997)) + list(range(65536, nblk))
    for b in blocks:
        ctr = (b // 65536, 0, b % 65536, 0)
        np.testing.assert_array_equal(O.philox(ctr, key), words[b])


def test_philox_all_counter_lanes_change_output():
    base = O.philox((1, 2, 3, 4), (5, 6))
    for lane in range(4):
        c = [1, 2, 3, 4]
        c[lane] ^= 1
        assert not np.array_equal(O.philox(c, (5, 6)), base)
    assert not np.array_equal(O.philox((1, 2, 3, 4), (5, 7)), base)


def test_uniform_is_exact_and_open():
    assert O.uniform(0, 0) == 2.0 ** -53
    assert O.uniform(0xFFFFFFFF, 0xFFFFFFFF) == 1.0 - 2.0 ** -53
    # 52 bits: the low 12 bits of the second word do not matter
    assert O.uniform(7, 0xABC) == O.uniform(7, 0)
    assert O.uniform(0, 1 << 12) == 1.5 * 2.0 ** -52
    assert O.uniform(1, 0) == (2.0 ** 20 + 0.5) * 2.0 ** -52


def test_draw_layout():
    p = I.small_multigroup(seed=0x1234567890)
    op = O.OracleProblem(p)
    pid, step = (5 << 44) | (77 << 20) | 3, 9
    key = (p.seed & 0xFFFFFFFF, (p.seed >> 32) ^ p.instance)
    for j in range(6):
        w = O.philox((pid & 0xFFFFFFFF, pid >> 32, step, j // 2), key)
        exp = O.uniform(w[0], w[1]) if j % 2 == 0 else O.uniform(w[2], w[3])
        assert O.draw(op, pid, step, j) == exp


def test_uniform_moments():
    rng_words = O.philox((0, 0, 0, 0), (1, 2))
    us = np.array([O.uniform(*O.philox((i, 0, 0, 0), (1, 2))[:2]) for i in range(20000)])
    assert rng_words.dtype == np.uint32
    assert abs(us.mean() - 0.5) < 4 * (1 / np.sqrt(12 * len(us)))
    assert abs(us.var() - 1 / 12) < 0.005


def test_identity_space_ends_at_step_2_pow_20():
    # a newborn's identity holds its birth step in 20 bits: the last step
    # that may sample is 2^20 - 1; the next samples nothing and says so
    # (otherwise its identities and random streams would repeat step 0's)
    p = I.small_multigroup(nx=12, G=4, omega_ref=1e-6)
    op = O.OracleProblem(p)
    st = O.initial_state(op)
    st, tal, _, status = O.step(op, st)
    assert status == 0 and tal.c.n_born > 100
    born0 = tal.c.n_born
    st.step = (1 << 20) - 1
    st1, tal, _, status = O.step(op, st)
    assert status == 0 and tal.c.n_born > 100
    assert (st1.particles.view()["id"] >> 44 == (1 << 20) - 1).sum() > 0
    st.step = 1 << 20
    st2, tal, _, status = O.step(op, st)
    assert status == O.OR_ERR_IDSPACE and tal.c.n_born == 0
    assert int(np.sum(tal.N)) == 0 and born0 > 0
