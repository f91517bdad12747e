"""Generate the oracle's table of hybrid Gauss-trapezoidal end corrections for
log-singular integrands (Alpert's rules, cited in Section 3.2 of the paper; the
paper does not print the nodes and weights).

Defining conditions (generalised Euler-Maclaurin expansion of the punctured
trapezoid sum at a singular end point): the rule
    h [ sum_{m=1}^{l} w_m f(x_m h) + sum_{k>=a} f(k h) ]
integrates x^g and x^g log x with no error term of order h^{g+1} for
g = 0..l-1, i.e.
    sum_m w_m x_m^g          = -zeta(-g, a)
    sum_m w_m x_m^g log x_m  =  zeta'(-g, a)        (derivative in s)
with zeta(s, a) the Hurwitz zeta function.  2l equations, 2l unknowns
(x_m in (0, a), w_m > 0).  Solved with mpmath Newton (findroot) at 40 digits,
by continuation in l with a = l, from a Gauss-Legendre start for l <= 3.

Run:  python -m oracle.gen_alpert_rules   (writes oracle/alpert_rules.json)
"""
import json
import os

import mpmath as mp

mp.mp.dps = 40
LMAX = 10


def residual_and_jacobian(l, a, x, w, zp, zl):
    F = []
    J = mp.zeros(2 * l, 2 * l)
    for g in range(l):
        F.append(mp.fsum(w[m] * x[m] ** g for m in range(l)) + zp[g])
        F.append(mp.fsum(w[m] * x[m] ** g * mp.log(x[m]) for m in range(l)) - zl[g])
        for m in range(l):
            xg = x[m] ** g
            dxg = g * x[m] ** (g - 1) if g > 0 else mp.mpf(0)
            lg = mp.log(x[m])
            J[2 * g, m] = w[m] * dxg
            J[2 * g, l + m] = xg
            J[2 * g + 1, m] = w[m] * (dxg * lg + xg / x[m])
            J[2 * g + 1, l + m] = xg * lg
    return mp.matrix(F), J


def solve(l, a, x0, w0, iters=300):
    """Damped Newton (backtracking on the residual norm) on the 2l conditions."""
    zp = [mp.zeta(-g, a) for g in range(l)]
    zl = [mp.zeta(-g, a, 1) for g in range(l)]
    x = [mp.mpf(v) for v in x0]
    w = [mp.mpf(v) for v in w0]
    F, J = residual_and_jacobian(l, a, x, w, zp, zl)
    nrm = mp.norm(F)
    for _ in range(iters):
        if nrm < mp.mpf(10) ** -32:
            break
        d = mp.lu_solve(J, -F)
        lam = mp.mpf(1)
        while lam > mp.mpf(10) ** -8:
            xn = [x[m] + lam * d[m] for m in range(l)]
            wn = [w[m] + lam * d[l + m] for m in range(l)]
            if all(v > 0 for v in xn):
                Fn, Jn = residual_and_jacobian(l, a, xn, wn, zp, zl)
                if mp.norm(Fn) < nrm:
                    break
            lam /= 2
        else:
            return None
        x, w, F, J, nrm = xn, wn, Fn, Jn, mp.norm(Fn)
    if nrm > mp.mpf(10) ** -30:
        return None
    order = sorted(range(l), key=lambda i: x[i])
    return [x[i] for i in order], [w[i] for i in order]


def main():
    rules = {}
    x, w = None, None
    for l in range(1, LMAX + 1):
        a = l
        if l <= 3:
            nodes, wts = zip(*[(mp.mpf(a) * (mp.mpf(i) + mp.mpf(1) / 2) / l, mp.mpf(a) / l) for i in range(l)])
            x0, w0 = list(nodes), list(wts)
            if l == 3:
                x0 = [mp.mpf("0.0649"), mp.mpf("0.6889"), mp.mpf("1.9155")]
                w0 = [mp.mpf("0.23"), mp.mpf("1.04"), mp.mpf("1.23")]
        else:
            # continuation from (l-1, a-1): stretch the nodes by a/(a-1), add one node near 0
            s = mp.mpf(a) / (a - 1)
            x0 = [mp.mpf(x[0]) * s / 8] + [xi * s for xi in x]
            w0 = [mp.mpf(w[0]) * s / 4] + [wi * s for wi in w]
        res = solve(l, a, x0, w0)
        if res is None and l > 3:
            s = mp.mpf(a) / (a - 1)
            for frac in [mp.mpf(1) / 16, mp.mpf(1) / 4, mp.mpf(1) / 2, mp.mpf(3) / 4, mp.mpf(1) / 32]:
                x0 = sorted([mp.mpf(x[0]) * s * frac] + [xi * s for xi in x])
                w0 = [mp.mpf(a) / l] * l
                res = solve(l, a, x0, w0)
                if res is not None:
                    break
        assert res is not None, l
        x, w = res
        assert all(0 < xi < a for xi in x) and all(wi > 0 for wi in w), (l, x, w)
        rules[str(l)] = {"l": l, "a": a, "nodes": [mp.nstr(v, 30) for v in x],
                         "weights": [mp.nstr(v, 30) for v in w]}
        print(l, a, [mp.nstr(v, 8) for v in x], flush=True)
    path = os.path.join(os.path.dirname(__file__), "alpert_rules.json")
    with open(path, "w") as fh:
        json.dump(rules, fh, indent=1)


if __name__ == "__main__":
    main()
