"""Test-only restatements of two of the paper's bit-parallel threshold
algorithms, over NumPy uint64 word arrays.  They exist to cross-check the
oracle from a different formulation; nothing in the product uses them.

* ``looped``: the Looped recurrence (Sec. 4.4, Algorithm "Looped"):
  C_j holds "at least j of the inputs seen so far"; each new input b
  updates C_j <- C_j OR (C_{j-1} AND b) for j from min(T, i) down to 2, then
  C_1 <- C_1 OR b.
* ``carry_save_vertical``: the scheduled carry-save vertical counter
  (Sec. 4.4, Algorithm "carry-save-vert", after Ellingsen): digits in
  {0, 1, 2} held as two bitmaps, inputs added on the schedule given by the
  trailing zeros of a time counter, then converted to binary and compared
  with T by adding the two's complement of T and reading the sign.
"""
from __future__ import annotations

import numpy as np

ALL = np.uint64(0xFFFFFFFFFFFFFFFF)


def looped(bitmaps: list[np.ndarray], T: int) -> np.ndarray:
    """Threshold T over the bitmaps by the Looped recurrence (1 <= T <= N)."""
    n = len(bitmaps)
    assert 1 <= T <= n
    C = [np.zeros_like(bitmaps[0]) for _ in range(T + 1)]  # C[1..T]
    C[1] = bitmaps[0].copy()
    for i in range(2, n + 1):
        b = bitmaps[i - 1]
        for j in range(min(T, i), 1, -1):
            C[j] = C[j] | (C[j - 1] & b)
        C[1] = C[1] | b
    return C[T]


def _trailing_zeros(t: int) -> int:
    x = 0
    while t % 2 == 0:
        t //= 2
        x += 1
    return x


def carry_save_vertical(bitmaps: list[np.ndarray], T: int) -> np.ndarray:
    """Threshold T by the scheduled carry-save counter; the algorithm states
    2 <= T < N, and the restatement is also exercised at other T."""
    n = len(bitmaps)
    L = 1 + (2 * n).bit_length() - 1  # 1 + floor(log2(2N)) digit pairs
    zero = np.zeros_like(bitmaps[0])
    C1 = [zero.copy() for _ in range(L + 2)]  # 1-based
    C2 = [zero.copy() for _ in range(L + 2)]
    t = 0
    for i in range(1, n + 1):
        c = bitmaps[i - 1]
        t += 1
        x = _trailing_zeros(t)
        for p in range(1, x + 1):
            a, b = C1[p], C2[p]
            C1[p] = zero.copy()
            s = a ^ b
            C2[p] = s ^ c
            c = (a & b) | (c & s)
        # the schedule never overwrites a live first digit
        assert not C1[x + 1].any(), "carry-save schedule overwrote a live digit"
        C1[x + 1] = c
    # redundant digits -> binary digits V_1 .. V_{L-1}
    V = [zero.copy() for _ in range(L + 1)]
    cin = zero.copy()
    for i in range(1, L):
        a, b = C1[i], C2[i]
        s = a ^ b
        V[i] = s ^ cin
        cin = (a & b) | (cin & s)
    assert not (cin | C1[L] | C2[L]).any(), "conversion left a carry"
    # add the two's complement of T over L bits; the top bit is the sign
    negT = (-T) & ((1 << L) - 1)
    cin = zero.copy()
    for i in range(1, L + 1):
        a = V[i]
        if (negT >> (i - 1)) & 1:
            s = ~a
            V[i] = s ^ cin
            cin = a | (cin & s)
        else:
            s = a
            V[i] = s ^ cin
            cin = cin & s
    return ~V[L]
