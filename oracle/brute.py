"""Brute-force occurrence list, pure Python -- TEST INFRASTRUCTURE ONLY.

The problem statement (Section 1) written out as loops: every pair (i, p)
with T[i..i+m) == P_p, 0-based, sorted by i then p.  Only for tiny inputs.
"""


def occurrences(T, P):
    T = bytes(T)
    P = [bytes(p) for p in P]
    out = []
    for i in range(len(T)):
        for p, pat in enumerate(P):
            m = len(pat)
            if m > 0 and i + m <= len(T) and T[i:i + m] == pat:
                out.append((i, p))
    out.sort()
    return out
