"""Writes appendix_min_k_distribution.txt: the distribution gamma(l, m, k) of the number m
of successive min-k elements met by a sequential scan of a random permutation of l
distinct keys, by the recurrence of the paper's Appendix (complexity analysis of the
k-selection), with alpha(n, k) = 1 for n <= k and k / n above, in exact fractions.

Run from the repository root:  python tests/golden/make_appendix_min_k.py
"""
import os
from fractions import Fraction

L_MAX, K_MAX = 7, 3


def alpha(n, k):
    return Fraction(1) if n <= k else Fraction(k, n)


def gamma(l, m, k, memo={}):
    key = (l, m, k)
    if key not in memo:
        if l == 0:
            memo[key] = Fraction(1) if m == 0 else Fraction(0)
        elif m == 0:
            memo[key] = Fraction(0)
        else:
            a = alpha(l, k)
            memo[key] = gamma(l - 1, m - 1, k) * a + gamma(l - 1, m, k) * (1 - a)
    return memo[key]


def main():
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "appendix_min_k_distribution.txt")
    with open(out, "w") as f:
        f.write("# gamma(l, m, k): probability that a sequential scan of a random permutation of l\n"
                "# distinct keys meets exactly m elements of the successive min-k (paper, Appendix:\n"
                "# complexity analysis of the k-selection; recurrence in gamma, alpha(n, k) = 1 for\n"
                "# n <= k, k/n above).  Columns: l k m numerator denominator.  Written by\n"
                "# tests/golden/make_appendix_min_k.py.\n")
        for l in range(1, L_MAX + 1):
            for k in range(1, min(K_MAX, l) + 1):
                for m in range(0, l + 1):
                    g = gamma(l, m, k)
                    if g:
                        f.write("%d %d %d %d %d\n" % (l, k, m, g.numerator, g.denominator))


if __name__ == "__main__":
    main()
