"""MurmurHash3 bodies written for the tests from the published algorithm
(Appleby's MurmurHash3_x86_32 and MurmurHash3_x64_128).  The finaliser is
passed in, so the oracle's fmix32/fmix64 can be checked against the published
vectors through the full hash."""

M32 = 0xFFFFFFFF
M64 = (1 << 64) - 1


def _rotl32(x, r):
    return ((x << r) | (x >> (32 - r))) & M32


def _rotl64(x, r):
    return ((x << r) | (x >> (64 - r))) & M64


def murmur3_x86_32(data: bytes, seed: int, fmix32) -> int:
    c1, c2 = 0xCC9E2D51, 0x1B873593
    h = seed & M32
    nblocks = len(data) // 4
    for b in range(nblocks):
        k = int.from_bytes(data[4 * b:4 * b + 4], "little")
        k = (k * c1) & M32
        k = _rotl32(k, 15)
        k = (k * c2) & M32
        h ^= k
        h = _rotl32(h, 13)
        h = (h * 5 + 0xE6546B64) & M32
    tail = data[4 * nblocks:]
    if tail:
        k = int.from_bytes(tail, "little")
        k = (k * c1) & M32
        k = _rotl32(k, 15)
        k = (k * c2) & M32
        h ^= k
    h ^= len(data)
    return fmix32(h)


def murmur3_x64_128(data: bytes, seed: int, fmix64) -> bytes:
    c1, c2 = 0x87C37B91114253D5, 0x4CF5AD432745937F
    h1 = h2 = seed & M64
    nblocks = len(data) // 16
    for b in range(nblocks):
        k1 = int.from_bytes(data[16 * b:16 * b + 8], "little")
        k2 = int.from_bytes(data[16 * b + 8:16 * b + 16], "little")
        k1 = (k1 * c1) & M64
        k1 = _rotl64(k1, 31)
        k1 = (k1 * c2) & M64
        h1 ^= k1
        h1 = _rotl64(h1, 27)
        h1 = (h1 + h2) & M64
        h1 = (h1 * 5 + 0x52DCE729) & M64
        k2 = (k2 * c2) & M64
        k2 = _rotl64(k2, 33)
        k2 = (k2 * c1) & M64
        h2 ^= k2
        h2 = _rotl64(h2, 31)
        h2 = (h2 + h1) & M64
        h2 = (h2 * 5 + 0x38495AB5) & M64
    tail = data[16 * nblocks:]
    if len(tail) > 8:
        k2 = int.from_bytes(tail[8:], "little")
        k2 = (k2 * c2) & M64
        k2 = _rotl64(k2, 33)
        k2 = (k2 * c1) & M64
        h2 ^= k2
    if tail:
        k1 = int.from_bytes(tail[:8], "little")
        k1 = (k1 * c1) & M64
        k1 = _rotl64(k1, 31)
        k1 = (k1 * c2) & M64
        h1 ^= k1
    h1 ^= len(data)
    h2 ^= len(data)
    h1 = (h1 + h2) & M64
    h2 = (h2 + h1) & M64
    h1 = fmix64(h1)
    h2 = fmix64(h2)
    h1 = (h1 + h2) & M64
    h2 = (h2 + h1) & M64
    return h1.to_bytes(8, "little") + h2.to_bytes(8, "little")


def smhasher_verification(hash_fn, nbytes: int) -> int:
    """SMHasher's VerificationTest: hash keys of length 0..255 (key[i] = i)
    with seed 256 - length, hash the concatenated digests with seed 0 and
    return the first four bytes little-endian."""
    digests = b""
    for n in range(256):
        digests += hash_fn(bytes(range(n)), 256 - n)[:nbytes]
    return int.from_bytes(hash_fn(digests, 0)[:4], "little")
