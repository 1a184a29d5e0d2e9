"""The closed form of a flip's change of F_2 (Eq. 4 with alpha = 2, the sum of squared
sidelobes) that the alpha = 2 neighbourhood kernel evaluates, and the bit-plane arithmetic it
evaluates it with, against recomputing F_2 after each flip (brute force, plain Python).

With C_k = sum_i s_i s_{i+k} (Eq. 2) and the flip of s_j (Sec. 3) changing C_k by
delta_k = -2 s_j (s_{j+k} + s_{j-k}) (terms outside the sequence absent):

    Delta F_2(j) = sum_{k>=1} (2 C_k delta_k + delta_k^2)
                 = -4 s_j (X_j + Y_j) + 4 (L - 1) + 8 Z_j,
    X_j = sum_{k=1}^{L-1-j} C_k s_{j+k},  Y_j = sum_{k=1}^{j} C_k s_{j-k},
    Z_j = sum_{k=1}^{min(j, L-1-j)} s_{j+k} s_{j-k}.

With x_i = (1 - s_i) / 2 the sequence's bits and C_k in two's complement over P planes
(C_k = sum_{p<P-1} 2^p c_{k,p} - 2^(P-1) c_{k,P-1}, P = bitlen(max |C_k|) + 1),
sum_k C_k x_{j+k} = sum_p w_p popcount(c_p AND x-window), so X_j = S(L-1-j) - 2 that sum
with S(K) = sum_{k=1}^K C_k, and likewise Y_j; Z_j = min(j, L-1-j) - 2 popcount of the
differing partner bits.
"""
import numpy as np
import pytest


def autocorr(s):
    L = len(s)
    return [sum(int(s[i]) * int(s[i + k]) for i in range(L - k)) for k in range(L)]


def energy(s):
    C = autocorr(s)
    return sum(c * c for c in C[1:])


def closed_form(s):
    L = len(s)
    C = autocorr(s)
    out = []
    for j in range(L):
        X = sum(C[k] * int(s[j + k]) for k in range(1, L - j))
        Y = sum(C[k] * int(s[j - k]) for k in range(1, j + 1))
        Z = sum(int(s[j + k]) * int(s[j - k]) for k in range(1, min(j, L - 1 - j) + 1))
        out.append(-4 * int(s[j]) * (X + Y) + 4 * (L - 1) + 8 * Z)
    return out


def bit_planes(s):
    """The kernel's arithmetic: planes of C over 32-bit words of shifts, windows of bits."""
    L = len(s)
    C = autocorr(s)
    x = [(1 - int(v)) // 2 for v in s]
    psl = max((abs(c) for c in C[1:]), default=0)
    P = psl.bit_length() + 1
    nw = (L - 1 + 31) // 32
    planes = [[0] * P for _ in range(nw)]
    for k in range(1, L):
        w, t = divmod(k - 1, 32)
        for p in range(P):
            if (C[k] >> p) & 1:  # Python's >> on negative ints is the two's-complement bit
                planes[w][p] |= 1 << t
    wt = [1 << p for p in range(P - 1)] + [-(1 << (P - 1))]
    S = [0] * L
    for k in range(1, L):
        S[k] = S[k - 1] + C[k]

    def xbit(i):
        return x[i] if 0 <= i < L else 0

    r = [x[L - 1 - i] for i in range(L)]  # the reversed bits: backward partners read forward

    def rbit(i):
        return r[i] if 0 <= i < L else 0

    out = []
    for j in range(L):
        kplus, kin = L - 1 - j, min(j, L - 1 - j)
        sx = sy = zd = 0
        for w in range(nw):
            fw = sum(xbit(j + 1 + 32 * w + t) << t for t in range(32))  # bit t: x_{j+k}, k = 1 + 32w + t
            rw = sum(xbit(j - 1 - 32 * w - t) << t for t in range(32))  # bit t: x_{j-k}
            assert rw == sum(rbit(L - j + 32 * w + t) << t for t in range(32))  # = r from L - j
            for p in range(P):
                sx += wt[p] * bin(planes[w][p] & fw).count("1")
                sy += wt[p] * bin(planes[w][p] & rw).count("1")
            lim = max(0, min(32, kin - 32 * w))
            zd += bin((fw ^ rw) & ((1 << lim) - 1)).count("1")
        X = S[kplus] - 2 * sx
        Y = S[j] - 2 * sy
        Z = kin - 2 * zd
        sj = 1 - 2 * x[j]
        out.append(-4 * sj * (X + Y) + 4 * (L - 1) + 8 * Z)
    return out


def brute(s):
    e0 = energy(s)
    out = []
    for j in range(len(s)):
        t = s.copy()
        t[j] = -t[j]
        out.append(energy(t) - e0)
    return out


@pytest.mark.parametrize("L", [2, 3, 5, 13, 31, 32, 33, 64, 65, 97])
def test_closed_form_matches_recomputed_energy(L):
    rng = np.random.default_rng(L)
    for _ in range(3):
        s = rng.choice(np.array([-1, 1], dtype=np.int64), size=L)
        want = brute(s)
        assert closed_form(s) == want
        assert bit_planes(s) == want


def test_closed_form_special_sequences():
    # all ones: C_k = L - k, the largest PSL (the sign plane and the widest planes);
    # Barker 13: every |C_k| <= 1; alternating: C_k = (-1)^k (L - k)
    for s in (np.ones(70, dtype=np.int64), np.array([1, 1, 1, 1, 1, -1, -1, 1, 1, -1, 1, -1, 1]),
              np.array([(-1) ** i for i in range(45)], dtype=np.int64)):
        want = brute(s)
        assert closed_form(s) == want
        assert bit_planes(s) == want


def test_barker13_is_a_local_optimum():
    # Barker 13 has E = 6, the lowest energy at L = 13: no flip lowers it
    s = np.array([1, 1, 1, 1, 1, -1, -1, 1, 1, -1, 1, -1, 1])
    assert energy(s) == 6
    assert min(closed_form(s)) > 0


def _fa(a, b, c):
    """Full adder over 32-bit slices: (sum, carry)."""
    return a ^ b ^ c, ((a & b) | (c & (a ^ b))) & 0xFFFFFFFF


def csa_count(words):
    """The kernel's carry-save count of the set bits of a list of 32-bit words: four words at a
    time into (ones, twos), the carries into the fours column counted per group; a short last
    group reads zero words."""
    ones = twos = fours = 0
    pad = words + [0] * (-len(words) % 4)
    for g in range(0, len(pad), 4):
        s1, c1 = _fa(ones, pad[g], pad[g + 1])
        s2, c2 = _fa(s1, pad[g + 2], pad[g + 3])
        ones = s2
        s4, c4 = _fa(twos, c1, c2)
        twos = s4
        fours += bin(c4).count("1")
    return bin(ones).count("1") + 2 * bin(twos).count("1") + 4 * fours


@pytest.mark.parametrize("n", [0, 1, 3, 4, 5, 8, 31, 32, 33, 128])
def test_carry_save_count_matches_popcount(n):
    rng = np.random.default_rng(n)
    for dense in (False, True):
        words = [int(w) for w in rng.integers(0, 1 << 32, size=n, dtype=np.uint64)]
        if dense:
            words = [0xFFFFFFFF] * n  # every column carries
        assert csa_count(words) == sum(bin(w).count("1") for w in words)
