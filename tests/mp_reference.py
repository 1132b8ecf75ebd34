"""Arbitrary-precision (mpmath, 50 digits) evaluation of the Berends-Giele
recursion of Sec. 3 (Eq. (BG-recursion) and its shorthand), used by the tests
only as an exact reference on the same FP64 inputs to measure how much
rounding error an FP64 evaluation of a given event can carry."""
import mpmath as mp


def _dot(a, b):
    return a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3]


def amp_exact(order, k, eps, dps=50):
    with mp.workdps(dps):
        L = len(order) - 1
        lk = [[mp.mpf(float(x)) for x in k[order[a + 1]]] for a in range(L)]
        le = [[mp.mpc(complex(x)) for x in eps[order[a + 1]]] for a in range(L)]
        J, K = {}, {}
        for a in range(L):
            J[(a, a)], K[(a, a)] = le[a], lk[a]
        num = None
        for ln in range(2, L + 1):
            for m in range(0, L - ln + 1):
                n = m + ln - 1
                K[(m, n)] = [K[(m, n - 1)][u] + lk[n][u] for u in range(4)]
                acc = [mp.mpc(0)] * 4
                for i in range(m, n):
                    Ja, Ka, Jb, Kb = J[(m, i)], K[(m, i)], J[(i + 1, n)], K[(i + 1, n)]
                    c1, c2, c3 = 2 * _dot(Ja, Kb), 2 * _dot(Jb, Ka), _dot(Ja, Jb)
                    acc = [acc[u] + c1 * Jb[u] - c2 * Ja[u] + c3 * (Ka[u] - Kb[u]) for u in range(4)]
                for i in range(m, n - 1):
                    for j in range(i + 1, n):
                        Ja, Jb, Jc = J[(m, i)], J[(i + 1, j)], J[(j + 1, n)]
                        ac, ab, cb = _dot(Ja, Jc), _dot(Ja, Jb), _dot(Jc, Jb)
                        acc = [acc[u] + 2 * ac * Jb[u] - ab * Jc[u] - cb * Ja[u] for u in range(4)]
                if ln < L:
                    K2 = _dot(K[(m, n)], K[(m, n)])
                    J[(m, n)] = [x / K2 for x in acc]
                else:
                    num = acc
        e0 = [mp.mpc(complex(x)) for x in eps[order[0]]]
        return complex(_dot(e0, num))
