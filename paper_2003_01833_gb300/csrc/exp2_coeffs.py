"""Coefficients of the float32 exp2 polynomial used by the Yukawa kernel.

2^f on [-1/2, 1/2] is approximated by a degree-6 polynomial whose relative
error equioscillates (Remez exchange algorithm, starting from Chebyshev
extrema).  Run this script to regenerate the constants printed into
interact.cu; it needs NumPy and mpmath (shipped with SymPy).
"""
import mpmath as mp

mp.mp.dps = 40
DEG = 6
A, B = mp.mpf(-0.5), mp.mpf(0.5)


def f(x):
    return mp.power(2, x)


def solve(xs):
    # p(x_i) + (-1)^i E f(x_i) = f(x_i): unknowns c_0..c_DEG, E (relative error)
    n = DEG + 2
    M = mp.matrix(n, n)
    rhs = mp.matrix(n, 1)
    for i, x in enumerate(xs):
        for j in range(DEG + 1):
            M[i, j] = x**j
        M[i, DEG + 1] = (-1) ** i * f(x)
        rhs[i] = f(x)
    sol = mp.lu_solve(M, rhs)
    return [sol[j] for j in range(DEG + 1)], sol[DEG + 1]


def rel_err(c, x):
    p = sum(cj * x**j for j, cj in enumerate(c))
    return (p - f(x)) / f(x)


def remez(iters=12):
    n = DEG + 2
    xs = [(A + B) / 2 + (B - A) / 2 * mp.cos(mp.pi * (n - 1 - i) / (n - 1)) for i in range(n)]
    for _ in range(iters):
        c, E = solve(xs)
        # new reference: extrema of the error between sign changes
        grid = [A + (B - A) * i / 4000 for i in range(4001)]
        errs = [rel_err(c, x) for x in grid]
        ext = []
        seg_start = 0
        for i in range(1, len(grid)):
            if mp.sign(errs[i]) != mp.sign(errs[seg_start]):
                j = max(range(seg_start, i), key=lambda t: abs(errs[t]))
                ext.append(grid[j])
                seg_start = i
        j = max(range(seg_start, len(grid)), key=lambda t: abs(errs[t]))
        ext.append(grid[j])
        if len(ext) >= n:
            # keep n alternating extrema with the largest magnitudes
            while len(ext) > n:
                if abs(rel_err(c, ext[0])) < abs(rel_err(c, ext[-1])):
                    ext.pop(0)
                else:
                    ext.pop()
            xs = ext
    c, E = solve(xs)
    return c, E


if __name__ == "__main__":
    c, E = remez()
    print("max relative error", mp.nstr(abs(E), 5))
    for j, cj in enumerate(c):
        print(f"c{j} = {mp.nstr(cj, 17)}")
