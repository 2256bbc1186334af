"""Oracle: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), the generator
of Calc 2 (Sec. V), written from its published definition.

TEST INFRASTRUCTURE ONLY (see the package header).

One call maps a 128-bit counter (c0, c1, c2, c3) and a 64-bit key (k0, k1)
to four 32-bit words by ten rounds of
    (c0, c1, c2, c3) <- (hi(M1*c2) ^ c1 ^ k0, lo(M1*c2),
                         hi(M0*c0) ^ c3 ^ k1, lo(M0*c0))
with the key bumped by the Weyl constants (W0, W1) between rounds.

Stream layout shared by both implementations (a published-definition
generator implemented twice, not shared code):
    counter = (sample lo32, sample hi32, graph id, draw block)
    key     = (seed lo32, seed hi32)
A uniform double in (0, 1) is made from two words:
    u = ((w0 >> 5) * 2^26 + (w1 >> 6) + 0.5) * 2^-53.

Pinned by the Known-Answer vectors published with the Random123 library
(tests/golden/philox4x32_10_kat.txt).
"""
import numpy as np

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """Scalar Python reference: ctr = 4 ints, key = 2 ints -> 4 ints."""
    c0, c1, c2, c3 = [int(x) & MASK for x in ctr]
    k0, k1 = [int(x) & MASK for x in key]
    for r in range(10):
        p0 = M0 * c0
        p1 = M1 * c2
        c0, c1, c2, c3 = ((p1 >> 32) ^ c1 ^ k0) & MASK, p1 & MASK, \
                         ((p0 >> 32) ^ c3 ^ k1) & MASK, p0 & MASK
        if r < 9:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
    return c0, c1, c2, c3


def philox_np(c0, c1, c2, c3, k0, k1):
    """Vectorised version over numpy uint64 arrays (values < 2^32)."""
    c0 = np.asarray(c0, np.uint64); c1 = np.asarray(c1, np.uint64)
    c2 = np.asarray(c2, np.uint64); c3 = np.asarray(c3, np.uint64)
    k0 = np.uint64(k0); k1 = np.uint64(k1)
    m = np.uint64(MASK)
    for r in range(10):
        p0 = np.uint64(M0) * c0
        p1 = np.uint64(M1) * c2
        n0 = ((p1 >> np.uint64(32)) ^ c1 ^ k0) & m
        n1 = p1 & m
        n2 = ((p0 >> np.uint64(32)) ^ c3 ^ k1) & m
        n3 = p0 & m
        c0, c1, c2, c3 = n0, n1, n2, n3
        if r < 9:
            k0 = (k0 + np.uint64(W0)) & m
            k1 = (k1 + np.uint64(W1)) & m
    return c0, c1, c2, c3


def uniforms(sample_idx, graph_id, seed, nblocks):
    """Uniform doubles for a vector of sample indices: shape (S, 2*nblocks);
    column 2b takes words (w0, w1) of draw block b, column 2b+1 (w2, w3)."""
    s = np.asarray(sample_idx, np.uint64)
    lo = s & np.uint64(MASK)
    hi = s >> np.uint64(32)
    out = np.empty((s.shape[0], 2 * nblocks))
    for b in range(nblocks):
        w = philox_np(lo, hi, np.full_like(s, graph_id), np.full_like(s, b),
                      seed & MASK, (seed >> 32) & MASK)
        for h in range(2):
            a = (w[2 * h] >> np.uint64(5)).astype(np.float64)
            c = (w[2 * h + 1] >> np.uint64(6)).astype(np.float64)
            out[:, 2 * b + h] = (a * 67108864.0 + c + 0.5) * (2.0 ** -53)
    return out


def uniforms_fine(sample_idx, graph_id, seed, nblocks):
    """The learned sampler's uniforms from the same words: the 52 high-order
    bits of (w0, w1) (all of w0, the top 20 of w1) form m, and
    u = (2m + 1) 2^-53 in (0, 1) (midpoint of the m-th cell of width 2^-52).
    Same layout as uniforms()."""
    s = np.asarray(sample_idx, np.uint64)
    lo = s & np.uint64(MASK)
    hi = s >> np.uint64(32)
    out = np.empty((s.shape[0], 2 * nblocks))
    for b in range(nblocks):
        w = philox_np(lo, hi, np.full_like(s, graph_id), np.full_like(s, b),
                      seed & MASK, (seed >> 32) & MASK)
        for h in range(2):
            m = (w[2 * h] << np.uint64(20)) | (w[2 * h + 1] >> np.uint64(12))
            out[:, 2 * b + h] = (2.0 * m.astype(np.float64) + 1.0) * (2.0 ** -53)
    return out
