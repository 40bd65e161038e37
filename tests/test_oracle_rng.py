"""Pins of the oracle's Philox4x32-10 (Salmon et al., SC'11).

The paper's Monte-Carlo block (Sec. II) states no generator; both sides use
counter-based Philox4x32-10.  The oracle's copy is pinned against NVIDIA's
host-side cuRAND Philox generator (a library routine, run on the CPU), whose
output block b is Philox of counter (b >> 16, 0, b & 0xffff, 0) under key
(seed low, seed high); that covers both key words and the counter words the
method uses (word 0 = particle, word 2 = 4*step + stream).
"""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O


def _curand():
    for name in ("libcurand.so.10", "libcurand.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            continue
    pytest.skip("libcurand not available")


def _curand_blocks(seed, first_block, nblocks):
    lib = _curand()
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), 161) == 0  # PHILOX4_32_10
    assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
    assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(4 * first_block)) == 0
    buf = np.zeros(4 * nblocks, dtype=np.uint32)
    assert lib.curandGenerate(gen, buf.ctypes.data_as(ctypes.c_void_p), ctypes.c_size_t(buf.size)) == 0
    lib.curandDestroyGenerator(gen)
    return buf.reshape(nblocks, 4)


@pytest.mark.parametrize("seed", [0, 1, 2, 0x123456789ABCDEF, 0xFFFFFFFFFFFFFFFF])
def test_philox_matches_curand_host_generator(seed):
    key = [seed & 0xFFFFFFFF, seed >> 32]
    # counter word 2 (4*step + stream) over the first blocks
    blocks = _curand_blocks(seed, 0, 64)
    for b in range(64):
        assert list(O.philox([0, 0, b, 0], key)) == list(blocks[b])
    # counter word 0 (particle index) and word 2 together, at larger offsets
    for pid, w2 in [(1, 0), (3, 5), (17, 4095), (1000, 65535), (123457, 33)]:
        blk = _curand_blocks(seed, (pid << 16) | w2, 1)[0]
        assert list(O.philox([pid, 0, w2, 0], key)) == list(blk)


def test_philox_words_are_uniform():
    # chi-square on the top 8 bits of 4*4096 words: a broken round function
    # (dropped multiply, wrong Weyl step) shows up as strong non-uniformity.
    words = np.concatenate([O.philox([i, 0, 7, 0], [1, 0]) for i in range(4096)])
    hist = np.bincount(words >> 24, minlength=256)
    expected = words.size / 256
    chi2 = ((hist - expected) ** 2 / expected).sum()
    assert 180 < chi2 < 340  # 255 dof, well inside +-4 sigma
