"""Pins of the oracle's Philox4x32-10 (Salmon et al., SC'11).

The paper's Monte-Carlo block (Sec. II) states no generator; both sides use
counter-based Philox4x32-10 with counter (particle, 0, 4*step + stream, 0)
under key (seed low, seed high).  The oracle's copy is pinned against two
library implementations run on the CPU:

* NVIDIA's host-side cuRAND Philox generator, whose output block b is Philox
  of counter (b >> 16, b >> 48, b & 0xffff, 0) under key (seed low, seed
  high): both key words and counter words 0-2;
* PyTorch's ATen `philox_engine` (a C++ header, compiled here into a small
  shim), whose counter is (offset low, offset high, subsequence low,
  subsequence high) under key (seed low, seed high): all four counter words
  and both key words with arbitrary values.
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


def _aten_shim(tmp_path_factory):
    """Compile a one-function shim around ATen's philox_engine with g++."""
    import os
    import shutil
    import subprocess
    try:
        import torch.utils.cpp_extension as ce
    except Exception:
        pytest.skip("torch headers not available")
    inc = [p for p in ce.include_paths() if os.path.exists(os.path.join(p, "ATen", "core", "PhiloxRNGEngine.h"))]
    gxx = shutil.which("g++")
    if not inc or not gxx:
        pytest.skip("g++ or ATen's PhiloxRNGEngine.h not available")
    d = tmp_path_factory.mktemp("aten_philox")
    src = d / "shim.cpp"
    src.write_text(
        "#include <ATen/core/PhiloxRNGEngine.h>\n"
        "#include <cstdint>\n"
        "extern \"C\" void aten_philox(const uint32_t c[4], const uint32_t k[2], uint32_t out[4]) {\n"
        "  at::philox_engine e(((uint64_t)k[1] << 32) | k[0], ((uint64_t)c[3] << 32) | c[2], 0);\n"
        "  e.set_offset(((uint64_t)c[1] << 32) | c[0]);\n"
        "  for (int i = 0; i < 4; ++i) out[i] = e();\n"
        "}\n")
    so = d / "shim.so"
    subprocess.run([gxx, "-O1", "-std=c++17", "-fPIC", "-shared", "-I", inc[0], str(src), "-o", str(so)], check=True)
    return ctypes.CDLL(str(so))


def test_philox_matches_aten_engine(tmp_path_factory):
    lib = _aten_shim(tmp_path_factory)
    rng = np.random.default_rng(11)
    cases = [([0, 0, 0, 0], [0, 0]), ([0xFFFFFFFF] * 4, [0xFFFFFFFF] * 2)]
    # arbitrary counters under key (0, 0) and under arbitrary keys
    for _ in range(200):
        c = [int(v) for v in rng.integers(0, 2 ** 32, size=4, dtype=np.uint64)]
        cases.append((c, [0, 0]))
        cases.append((c, [int(v) for v in rng.integers(0, 2 ** 32, size=2, dtype=np.uint64)]))
    for c, k in cases:
        ca, ka = np.array(c, np.uint32), np.array(k, np.uint32)
        out = np.zeros(4, np.uint32)
        lib.aten_philox(ca.ctypes.data, ka.ctypes.data, out.ctypes.data)
        assert list(O.philox(c, k)) == list(out), (c, k)
