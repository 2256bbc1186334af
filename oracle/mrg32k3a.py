"""Oracle: MRG32k3a (P. L'Ecuyer, "Good parameters and implementations for
combined multiple recursive random number generators", Operations Research
47 (1999)), the generator of Calc 1 (Sec. V), written from its published
definition in exact integer arithmetic.

TEST INFRASTRUCTURE ONLY (see the package header).

Two recursions
    x1_n = (1403580 x1_{n-2} - 810728 x1_{n-3}) mod m1,  m1 = 2^32 - 209,
    x2_n = (527612 x2_{n-1} - 1370589 x2_{n-3}) mod m2,  m2 = 2^32 - 22853,
output z_n = (x1_n - x2_n) mod m1.  As 3x3 matrices on the state vectors
(x_{n-3}, x_{n-2}, x_{n-1}) the steps are A1 and A2; a jump of k outputs is
A^k mod m, computed by squaring.

Stream layout (the paper gives none; reading, implemented twice):
    default state x1 = x2 = (12345, 12345, 12345);
    sample i of graph g under seed s starts at output position
        s * 2^96 + g * 2^80 + 64 i,
    and its draw block b (b = 0..M-1) takes the four outputs 4b .. 4b+3,
    mapped to two uniforms exactly as the Philox words are:
        u = ((w0 >> 5) * 2^26 + (w1 >> 6) + 0.5) * 2^-53.
"""
import numpy as np

M1 = 4294967087
M2 = 4294944443
A1 = ((0, 1, 0), (0, 0, 1), (M1 - 810728, 1403580, 0))
A2 = ((0, 1, 0), (0, 0, 1), (M2 - 1370589, 0, 527612))
SEED = (12345, 12345, 12345)


def step(s1, s2):
    """One output: new states and z (states are 3-tuples, oldest first)."""
    x1 = (1403580 * s1[1] - 810728 * s1[0]) % M1
    x2 = (527612 * s2[2] - 1370589 * s2[0]) % M2
    s1 = (s1[1], s1[2], x1)
    s2 = (s2[1], s2[2], x2)
    return s1, s2, (x1 - x2) % M1


def matmul(A, B, m):
    return tuple(tuple(sum(A[i][k] * B[k][j] for k in range(3)) % m for j in range(3)) for i in range(3))


def matvec(A, v, m):
    return tuple(sum(A[i][k] * v[k] for k in range(3)) % m for i in range(3))


def matpow(A, k, m):
    R = ((1, 0, 0), (0, 1, 0), (0, 0, 1))
    P = A
    while k:
        if k & 1:
            R = matmul(R, P, m)
        P = matmul(P, P, m)
        k >>= 1
    return R


def state_at(pos):
    """States after `pos` outputs from the default state (jump-ahead)."""
    return matvec(matpow(A1, pos, M1), SEED, M1), matvec(matpow(A2, pos, M2), SEED, M2)


def words(pos, count):
    """Outputs pos+1 .. pos+count (the outputs generated after `pos`)."""
    s1, s2 = state_at(pos)
    out = []
    for _ in range(count):
        s1, s2, z = step(s1, s2)
        out.append(z)
    return out


def uniforms(sample_idx, graph_id, seed, nblocks):
    """Uniform doubles (S, 2*nblocks), the same layout as philox.uniforms."""
    s = np.asarray(sample_idx, dtype=np.uint64)
    out = np.empty((s.shape[0], 2 * nblocks))
    base = (int(seed) << 96) + (int(graph_id) << 80)
    for r, i in enumerate(s):
        w = words(base + 64 * int(i), 4 * nblocks)
        for b in range(nblocks):
            for h in range(2):
                a = float(w[4 * b + 2 * h] >> 5)
                c = float(w[4 * b + 2 * h + 1] >> 6)
                out[r, 2 * b + h] = (a * 67108864.0 + c + 0.5) * (2.0 ** -53)
    return out
