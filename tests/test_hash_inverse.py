"""The device code's inverse of the MurmurHash3 32-bit finaliser (fmix32_inv in
csrc/hg_device.cuh).  The partitioned build moves 32-bit keys as their hashes
h = fmix32(k ^ seed) and writes each key back as fmix32_inv(h) ^ seed, so the
table's keys are right only if fmix32_inv undoes fmix32 on every word.

Checked here without a GPU: the constants in the device function are the
inverses mod 2^32 of the finaliser's two published multipliers, and the
function's steps, applied to the oracle's fmix32 of sampled words (edge words
and 2^12 seeded random ones), give every word back."""
import pathlib
import re

import numpy as np

import oracle

SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2104_00792_gb300" / "csrc" / "hg_device.cuh"

# MurmurHash3_x86_32's finaliser multipliers (Appleby's reference code)
C1, C2 = 0x85EBCA6B, 0xC2B2AE35
M32 = (1 << 32) - 1


def _inv_body() -> str:
    m = re.search(r"uint32_t fmix32_inv\(uint32_t h\) \{(.*?)\n\}", SRC.read_text(), re.S)
    assert m, "fmix32_inv not found in the device header"
    return m.group(1)


def _inv_constants():
    return [int(c, 16) for c in re.findall(r"0x([0-9a-fA-F]+)u", _inv_body())]


def test_inverse_constants_undo_the_multipliers():
    consts = _inv_constants()
    assert len(consts) == 2
    # the device function multiplies by C2's inverse first, then by C1's
    assert (consts[0] * C2) & M32 == 1
    assert (consts[1] * C1) & M32 == 1


def test_inverse_steps_round_trip_the_oracle_hash():
    body = _inv_body()
    steps = [ln.strip() for ln in body.splitlines() if ln.strip().startswith("h ")]
    a, b = _inv_constants()
    assert steps == ["h ^= h >> 16;", f"h *= 0x{a:08x}u;", "h ^= (h >> 13) ^ (h >> 26);",
                     f"h *= 0x{b:08x}u;", "h ^= h >> 16;"]

    def inv(h: int) -> int:
        h ^= h >> 16
        h = (h * a) & M32
        h ^= (h >> 13) ^ (h >> 26)
        h = (h * b) & M32
        h ^= h >> 16
        return h

    rng = np.random.default_rng(0x210400792)
    words = [0, 1, 2, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFE, M32] + [int(x) for x in
                                                                  rng.integers(0, 1 << 32, 4096, dtype=np.uint64)]
    for x in words:
        assert inv(oracle.fmix32(x)) == x, hex(x)
