"""Coefficients of the sin/cos polynomials of sincos_pi (kc_device.cuh).

Minimax (Remez exchange) fits of the absolute error on [0, pi/2], in 40-digit
arithmetic (mpmath):

    sin r ~ r + r^3 (c3 + c5 r^2 + c7 r^4 + c9 r^6)            (odd, degree 9)
    cos r ~ 1 + r^2 (c2 + c4 r^2 + c6 r^4 + c8 r^6 + c10 r^8)  (even, degree 10)

The fits reach 4.6e-9 (sin) and 2.4e-10 (cos), below single-precision
rounding near 1; the coefficients are then rounded to float.  Run
`python minimax_sincos.py` to print them (about a minute and a half).
"""
import mpmath as mp

mp.mp.dps = 40


def remez(f, fixed, powers, a, b, iters=30, grid=20000):
    """Coefficients c_i of sum_i c_i x^powers[i] minimising the largest
    |f(x) - fixed(x) - sum_i c_i x^powers[i]| over [a, b] (Remez exchange:
    solve for equal alternating error on a reference set, move the reference
    to the extrema of the error on a dense grid, repeat)."""
    n = len(powers)
    ref = [a + (b - a) * (1 - mp.cos(mp.pi * k / n)) / 2 for k in range(n + 1)]
    xs = [a + (b - a) * mp.mpf(k) / grid for k in range(grid + 1)]
    c, err = None, None
    for _ in range(iters):
        A = mp.matrix(n + 1, n + 1)
        rhs = mp.matrix(n + 1, 1)
        for k, x in enumerate(ref):
            for i, p in enumerate(powers):
                A[k, i] = x ** p
            A[k, n] = (-1) ** k
            rhs[k] = f(x) - fixed(x)
        sol = mp.lu_solve(A, rhs)
        c = [sol[i] for i in range(n)]
        err = [f(x) - fixed(x) - sum(ci * x ** p for ci, p in zip(c, powers)) for x in xs]
        ext = [0] + [k for k in range(1, len(xs) - 1)
                     if (err[k] - err[k - 1]) * (err[k + 1] - err[k]) <= 0] + [len(xs) - 1]
        alt = []
        for k in ext:
            x, e = xs[k], err[k]
            if alt and mp.sign(e) == mp.sign(alt[-1][1]):
                if abs(e) > abs(alt[-1][1]):
                    alt[-1] = (x, e)
            else:
                alt.append((x, e))
        while len(alt) > n + 1:
            alt.pop(0 if abs(alt[0][1]) < abs(alt[-1][1]) else -1)
        if len(alt) < n + 1:
            break
        ref = [x for x, _ in alt]
    return c, max(abs(e) for e in err)


def main():
    half_pi = mp.pi / 2
    cs, es = remez(mp.sin, lambda x: x, [3, 5, 7, 9], mp.mpf("1e-4"), half_pi)
    cc, ec = remez(mp.cos, lambda x: 1, [2, 4, 6, 8, 10], mp.mpf(0), half_pi)
    print(f"// sin: max error {mp.nstr(es, 3)} on [0, pi/2]")
    for p, v in zip([3, 5, 7, 9], cs):
        print(f"constexpr float kSinC{p} = {mp.nstr(v, 12)}f;")
    print(f"// cos: max error {mp.nstr(ec, 3)} on [0, pi/2]")
    for p, v in zip([2, 4, 6, 8, 10], cc):
        print(f"constexpr float kCosC{p} = {mp.nstr(v, 12)}f;")


if __name__ == "__main__":
    main()
