"""Exact rational helpers for the tests: integer cube roots and the
continued-fraction convergents of a cube root (values closer to an irrational
window edge than double rounding resolves)."""


def icbrt(n):
    """Largest integer x with x^3 <= n (bisection on exact integers)."""
    lo, hi = 0, 1
    while hi ** 3 <= n:
        hi *= 2
    while hi - lo > 1:
        mid = (lo + hi) // 2
        if mid ** 3 <= n:
            lo = mid
        else:
            hi = mid
    return lo


def cube_root_convergents(a, count, digits=60):
    """Continued-fraction convergents p/q of the real cube root of the integer
    a (|p/q - a^(1/3)| < 1/q^2).  They are those of the rational
    floor(a^(1/3) 10^digits) / 10^digits while q stays far below 10^(digits/2)."""
    num, den = icbrt(a * 10 ** (3 * digits)), 10 ** digits
    out, (p0, q0, p1, q1) = [], (0, 1, 1, 0)
    while den and len(out) < count:
        m, (num, den) = num // den, (den, num % den)
        p0, q0, p1, q1 = p1, q1, m * p1 + p0, m * q1 + q0
        if q1 > 10 ** (digits // 2 - 5):
            break
        out.append((p1, q1))
    return out
