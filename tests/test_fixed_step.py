"""The fixed-point form of the path steps (Sec. II-B) against the error-term
form, in exact integer arithmetic: after i steps the error term has taken
floor((ns + 2 i dmin) / (2 ns)) minor steps; the fixed-point walk takes the
carries of 2^31 + i S.  Every slope S with 0 < S - dmin 2^32 / ns < 4610 (and
S = 2^32 - 1 for dmin = ns) must give the same steps for every ns <= 512."""
import numpy as np

MAX_NS = 512
EPS = 4610


def minor_steps_error_term(ns, d, i):
    return (ns + 2 * d * i) // (2 * ns)


def minor_steps_fixed_point(S, i):
    return (2**31 + i * S) >> 32


def slopes(ns, d):
    """The extreme valid slopes for each dmin in d (int64 arrays)."""
    lo = (d << 32) // ns + 1          # the least integer above d 2^32 / ns
    hi = ((d << 32) + ns - 1) // ns + EPS - 1   # the largest below d 2^32 / ns + EPS
    full = d == ns
    lo = np.where(full, 2**32 - 1, lo)
    hi = np.where(full, 2**32 - 1, hi)
    return lo, hi


def check_ns(ns):
    d = np.arange(ns + 1, dtype=np.int64)[:, None]
    i = np.arange(ns + 1, dtype=np.int64)[None, :]
    ref = minor_steps_error_term(ns, d, i)
    lo, hi = slopes(ns, d)
    assert np.all((lo < 2**32) & (hi < 2**32))
    for S in (lo, hi):
        got = minor_steps_fixed_point(S, i)
        bad = np.argwhere(got != ref)
        assert bad.size == 0, (ns, bad[:3])


def test_every_ns_up_to_512():
    for ns in range(1, MAX_NS + 1):
        check_ns(ns)


def test_bound_is_needed():
    """Far past the bound the same excess breaks a tie: the check above is
    not vacuous."""
    ns, d = 4096, 1365
    i = np.arange(ns + 1, dtype=np.int64)
    ref = minor_steps_error_term(ns, d, i)
    S = ((d << 32) + ns - 1) // ns + EPS - 1
    assert np.any(minor_steps_fixed_point(S, i) != ref)


def test_error_term_walk_matches_formula():
    """The closed form used above is the error-term walk itself."""
    rng = np.random.default_rng(3)
    for _ in range(200):
        ns = int(rng.integers(1, 600))
        d = int(rng.integers(0, ns + 1))
        e, m = ns, 0
        for k in range(ns + 1):
            assert m == minor_steps_error_term(ns, d, k)
            e += 2 * d
            if e >= 2 * ns:
                e -= 2 * ns
                m += 1
