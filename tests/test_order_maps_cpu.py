"""The index identities behind the kernels' ordered stores, checked on the CPU.

Sequency order stores dyadic output p at s = gray^{-1}(p), the s with s ^ (s >> 1) = p
(row s of the sequency-ordered matrix has s sign changes).  The kernels never compute
gray^{-1} of a whole position per element; they rely on these decompositions, checked here
for every position of signals up to 2^16 against a table built from the definition:

  * single-CTA tiles: an aligned 4-element chunk stays together, p = 4h + e goes to
    4 gray^{-1}(h) + (e-th entry of {0, 1, 3, 2}, or of {3, 2, 0, 1} when h has odd parity);
  * tensor-memory kernel: p = rho 2^L + 64 q + 4 c + e (L = m - 8) goes to run
    gray^{-1}(rho), 64-word segment gray^{-1}(q) complemented when that run is odd, 4-word
    group gray^{-1}(c) complemented when parity(q) differs from the run's parity, and
    word e reordered by parity(c) against that;
  * natural order is the bit reversal of the dyadic position (y_nat[k] = y[bitrev(k)]),
    so for the split Y = H_b X^T H_a the natural position of the dyadic output
    (k_lo 2^a + k_hi) is bitrev_b(k_lo) + 2^b bitrev_a(k_hi): rows of the first pass can
    keep natural order and the column tiles write stride-2^b runs.
"""

import numpy as np
import pytest


def ginv_table(n):
    t = np.zeros(n, dtype=np.int64)
    s = np.arange(n, dtype=np.int64)
    t[s ^ (s >> 1)] = s
    return t


def parity(x):
    return bin(int(x)).count("1") & 1


def bitrev(x, bits):
    r = 0
    for i in range(bits):
        r |= ((x >> i) & 1) << (bits - 1 - i)
    return r


@pytest.mark.parametrize("m", [2, 5, 8, 12, 16])
def test_fused_sequency_chunk_rule(m):
    n = 1 << m
    g = ginv_table(n)
    even, odd = (0, 1, 3, 2), (3, 2, 0, 1)
    for p in range(n):
        h, e = p >> 2, p & 3
        want = 4 * g[h] + (odd if parity(h) else even)[e]
        assert g[p] == want, p


@pytest.mark.parametrize("m", [15, 16])
def test_tensor_memory_sequency_decomposition(m):
    n, L = 1 << m, m - 8
    g = ginv_table(n)
    g256, g16, gq = ginv_table(256), ginv_table(16), ginv_table(1 << (L - 6))
    qmask = (1 << (L - 6)) - 1
    for p in range(n):
        rho, q, c, e = p >> L, (p >> 6) & qmask, (p >> 2) & 15, p & 3
        dr = int(g256[rho])
        pd = dr & 1
        qd = int(gq[q]) ^ (qmask if pd else 0)
        fx = parity(q) ^ pd
        C = int(g16[c]) ^ (15 if fx else 0)
        # the group's four words: (w0, w1, w3, w2), or (w2, w3, w1, w0) when parity(c) ^ fx
        order = (2, 3, 1, 0) if parity(c) ^ fx else (0, 1, 3, 2)
        slot = order.index(e)
        want = (dr << L) + 64 * qd + 4 * C + slot
        assert g[p] == want, p


@pytest.mark.parametrize("a,b", [(1, 1), (3, 5), (6, 4), (2, 9)])
def test_natural_order_of_the_split(a, b):
    m = a + b
    for klo in range(1 << b):
        for khi in range(1 << a):
            d = (klo << a) + khi  # dyadic position: row bitrev of the pass-1 label bits first
            assert bitrev(d, m) == bitrev(klo, b) + (bitrev(khi, a) << b)
