"""Brute-force checks written from the definitions, independent of the oracle's
algorithms: exact-rational steepest descent, path walking, dense solves."""
from fractions import Fraction

import numpy as np

# neighbour offsets (dx, dy) in ascending address order (k = 0..7)
NBR = [(-1, -1), (0, -1), (1, -1), (-1, 0), (1, 0), (-1, 1), (0, 1), (1, 1)]


def exact_gt(da, diag_a, db, diag_b):
    """Exact test da/dist_a > db/dist_b for positive rationals da, db, where
    dist is 1 (cardinal) or sqrt(2) (diagonal); sqrt(2) handled by squaring."""
    if diag_a == diag_b:
        return da > db
    if not diag_a and diag_b:      # da > db / sqrt2  <=>  2 da^2 > db^2
        return 2 * da * da > db * db
    return da * da > 2 * db * db   # da / sqrt2 > db  <=>  da^2 > 2 db^2


def exact_receivers(h):
    """Steepest strictly-downhill neighbour in exact rational arithmetic,
    lowest k on exact ties; perimeter and cells with no lower neighbour -> self."""
    ny, nx = h.shape
    rec = np.arange(nx * ny, dtype=np.int64)
    for y in range(1, ny - 1):
        for x in range(1, nx - 1):
            hc = Fraction(float(h[y, x]))
            best = None
            for k, (ox, oy) in enumerate(NBR):
                d = hc - Fraction(float(h[y + oy, x + ox]))
                if d <= 0:
                    continue
                diag = ox != 0 and oy != 0
                if best is None or exact_gt(d, diag, best[0], best[1]):
                    best = (d, diag, k)
            if best is not None:
                ox, oy = NBR[best[2]]
                rec[y * nx + x] = (y + oy) * nx + (x + ox)
    return rec


def exact_slope(h, c, n):
    """Exact slope (as a float from the exact rational, and sqrt) from c to n."""
    ny, nx = h.shape
    d = Fraction(float(h.flat[c])) - Fraction(float(h.flat[n]))
    diag = (c % nx != n % nx) and (c // nx != n // nx)
    return float(d) / (2 ** 0.5 if diag else 1.0)


def walk_to_sink(rec, c, limit):
    path = [c]
    while rec[c] != c:
        c = int(rec[c])
        path.append(c)
        if len(path) > limit:
            raise AssertionError("receiver graph has a cycle")
    return path


def path_counts(rec):
    """cnt[c] = number of cells whose receiver path passes through c."""
    n = rec.size
    cnt = np.zeros(n, np.int64)
    for c in range(n):
        for v in walk_to_sink(rec, c, n + 1):
            cnt[v] += 1
    return cnt


def is_perimeter(nx, ny, c):
    x, y = c % nx, c // nx
    return x == 0 or y == 0 or x == nx - 1 or y == ny - 1


def implicit_solve(h, rec, cnt, dx, K, m, U, dt, area_scale, Ufield=None):
    """The n = 1 implicit step as one dense linear system, independent of any
    ordering: (1+F_c) h'_c - F_c h'_r = h_c + dt U_c for eroding cells,
    h'_c = h_c + dt U_c for interior pits, h'_c = h_c on the perimeter."""
    ny, nx = h.shape
    n = nx * ny
    M = np.zeros((n, n))
    b = np.zeros(n)
    hf = h.ravel()
    for c in range(n):
        u = U if Ufield is None else Ufield.flat[c]
        if is_perimeter(nx, ny, c):
            M[c, c] = 1.0
            b[c] = hf[c]
        elif rec[c] == c:
            M[c, c] = 1.0
            b[c] = hf[c] + dt * u
        else:
            r = int(rec[c])
            diag = (c % nx != r % nx) and (c // nx != r // nx)
            d = dx * (2 ** 0.5 if diag else 1.0)
            F = K * dt * (cnt[c] * area_scale) ** m / d
            M[c, c] = 1.0 + F
            M[c, r] = -F
            b[c] = hf[c] + dt * u
    return np.linalg.solve(M, b).reshape(ny, nx)
