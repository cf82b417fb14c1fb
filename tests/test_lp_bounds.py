"""Soundness of the running error bounds behind the certified binary32 pivots
of the small-neighbourhood LP (k_lp_small32 in csrc/vrm_lp.cu).

The kernel keeps the 5 x 8 phase-I tableau of Sec. 4.1 (rows (1,0) (0,1)
(2,0) (1,1) (0,2), b = (0, 0, 2, 0, 2)) in binary32 together with, for every
entry, a bound E on its distance from the exact rational tableau of the same
pivot sequence started from the FP64 Vandermonde matrix, and takes a pivot
decision only where the binary32 value is farther than 1.25 E from the
tolerance.  These tests restate the kernel's update formulas in numpy
binary32 (a fused multiply-add as an exact binary64 product and sum rounded
to binary32), replay the same pivots in exact rational arithmetic
(fractions.Fraction), and check on random neighbourhoods that

* every binary32 entry lies within its bound of the exact value (the factor
  1.0001 covers the emulated fma's double rounding, at most 2^-53 on top of
  the binary32 rounding the bound accounts for);
* every certified decision is the exact decision;
* a row whose eligibility is uncertain is passed over only where, were it
  eligible, its exact ratio would lie above the exact tie limit (so that the
  leaving row is the same either way); binary-exact lattice columns, whose
  exact zeros carry running bounds, exercise that rule.
"""
from fractions import Fraction

import numpy as np

f32 = np.float32
U = f32(2.0 ** -24)
RCP_MUL = f32(3.01) * U
INIT = f32(1.0)  # scale of the initial conversion bounds (1 in the kernel)
TP_HI, TP_LO = f32(1.0000001e-9), f32(0.99999994e-9)
TS_HI, TS_LO = f32(1.0000001e-11), f32(0.99999994e-11)
TT_HI = f32(1.0000001e-12)
SAFE = f32(1.25)
STATS = {"uncertain_rows_passed": 0, "uncertain_rows_eligible": 0}
M, K = 5, 8
B = [0, 0, 2, 0, 2]


def fma32(a, b, c):
    return f32(np.float64(a) * np.float64(b) + np.float64(c))


def vcol64(xi, eta):
    return [xi, eta, xi * xi, xi * eta, eta * eta]


def columns(rng, R=2.0, r=0.5):
    """Eight annulus offsets (one per 45-degree segment, jittered), sorted by
    distance; FP64 offsets in units of h and their binary32 images
    f32(dx) * f32(1/h) with h = 2e-3, as the kernel forms them."""
    h = 2e-3
    ang = (np.arange(8) + rng.uniform(0.05, 0.95, 8)) * (np.pi / 4)
    rad = rng.uniform(r, R, 8)
    dx = np.array([np.float64(h) * rad[k] * np.cos(ang[k]) for k in range(8)])
    dy = np.array([np.float64(h) * rad[k] * np.sin(ang[k]) for k in range(8)])
    order = np.argsort(dx * dx + dy * dy, kind="stable")
    dx, dy = dx[order], dy[order]
    inv_h = 1.0 / h
    xi64, eta64 = dx * inv_h, dy * inv_h
    inv_h32 = f32(inv_h)
    xs = [f32(f32(dx[k]) * inv_h32) for k in range(8)]
    es = [f32(f32(dy[k]) * inv_h32) for k in range(8)]
    return xi64, eta64, xs, es


def lattice_columns(rng, R=2.0, r=0.5):
    """Eight offsets on the integer lattice of a binary-exact spacing
    h = 1/64 (one per 45-degree segment where the annulus has one), sorted by
    distance: the offsets, their products and many tableau entries are exact
    in binary32, and exact zeros appear after the first pivots."""
    pts = [(a, b) for a in range(-2, 3) for b in range(-2, 3) if r * r <= a * a + b * b <= R * R]
    segs = {}
    for a, b in pts:
        s_ = int(np.floor(np.arctan2(b, a) / (np.pi / 4))) % 8
        segs.setdefault(s_, []).append((a, b))
    chosen = [segs[k][rng.integers(len(segs[k]))] for k in sorted(segs)]
    while len(chosen) < 8:
        chosen.append(pts[rng.integers(len(pts))])
    h = 1.0 / 64
    dx = np.array([a * h for a, b in chosen])
    dy = np.array([b * h for a, b in chosen])
    order = np.argsort(dx * dx + dy * dy, kind="stable")
    dx, dy = dx[order], dy[order]
    xi64, eta64 = dx / h, dy / h
    xs = [f32(f32(dx[k]) * f32(1 / h)) for k in range(8)]
    es = [f32(f32(dy[k]) * f32(1 / h)) for k in range(8)]
    return xi64, eta64, xs, es


def run(xi64, eta64, xs, es, check):
    """The kernel's binary32 pivots with bounds; exact replay alongside.
    Returns the number of pivots taken before the end or an uncertain step."""
    V = [vcol64(xi64[k], eta64[k]) for k in range(K)]
    Tx = [[Fraction(V[k][r]) for k in range(K)] for r in range(M)]
    rx = [Fraction(b) for b in B]
    dx_ = [-sum(Tx[r][k] for r in range(M)) for k in range(K)]
    T = [[None] * K for _ in range(M)]
    E = [[None] * K for _ in range(M)]
    d, Ed = [None] * K, [None] * K
    for k in range(K):
        v = [xs[k], es[k], f32(xs[k] * xs[k]), f32(xs[k] * es[k]), f32(es[k] * es[k])]
        s = f32(0)
        sa = f32(0)
        se = f32(0)
        for r in range(M):
            T[r][k] = v[r]
            E[r][k] = f32(INIT * (f32(3.01) if r < 2 else f32(7.01)) * U * abs(v[r]))
            s = f32(s + v[r])
            sa = f32(sa + abs(v[r]))
            se = f32(se + E[r][k])
        d[k] = -s
        Ed[k] = fma32(f32(4.01) * U, sa, se)
    rhs = [f32(b) for b in B]
    Eb = [f32(0)] * M
    basis = list(range(M))
    basic = [False] * K
    n_art, it = M, 0

    def sound():
        for r in range(M):
            for k in range(K):
                check(abs(Fraction(float(T[r][k])) - Tx[r][k]) <= Fraction(float(E[r][k])) * Fraction(10001, 10000))
            check(abs(Fraction(float(rhs[r])) - rx[r]) <= Fraction(float(Eb[r])) * Fraction(10001, 10000))
        for k in range(K):
            if not basic[k]:
                check(abs(Fraction(float(d[k])) - dx_[k]) <= Fraction(float(Ed[k])) * Fraction(10001, 10000))

    sound()
    while n_art and it < 64:
        yes, un = [], []
        for k in range(K):
            if basic[k]:
                continue
            mg = f32(1.25) * Ed[k]
            if d[k] < -TP_HI - mg:
                yes.append(k)
            elif not d[k] > -TP_LO + mg:
                un.append(k)
        if not yes:
            return it
        q = yes[0]
        if any(k < q for k in un):
            return it
        # certified entering decision: the exact reduced costs agree
        check(dx_[q] < Fraction(-1, 10 ** 9))
        for k in range(q):
            if not basic[k]:
                check(dx_[k] >= Fraction(-1, 10 ** 9))
        a = [T[r][q] for r in range(M)]
        ea = [E[r][q] for r in range(M)]
        elig, amb = [], []
        for r in range(M):
            mg = SAFE * ea[r]
            mb = SAFE * Eb[r]
            nzr = rhs[r] > TS_HI + mb
            if a[r] > TP_HI + mg:
                elig.append(r)
                if not (nzr or rhs[r] < TS_LO - mb):
                    return it
            elif not a[r] < TP_LO - mg:
                # eligibility uncertain: the LP goes on only if the basic
                # value is certainly positive (and the ratio bound below holds)
                if not nzr:
                    return it
                amb.append(r)
        for r in range(M):
            if r not in amb:
                check((Tx[r][q] > Fraction(1, 10 ** 9)) == (r in elig))
        if not elig:
            return it
        if amb:
            # the largest possible tie limit from the binary32 ratio intervals
            # of the certainly eligible rows, as the kernel bounds it
            thhi = f32(3.0e38)
            for r in elig:
                nz = rhs[r] > TS_HI + SAFE * Eb[r]
                inv = f32(f32(1) / a[r])
                ratio = f32(rhs[r] * inv) if nz else f32(0)
                g = f32(ea[r] * inv)
                gg = fma32(f32(2) * g, g, g)
                if nz and not g <= 0.5:
                    return it
                er = f32(SAFE * fma32(RCP_MUL, ratio, f32(fma32(gg, f32(rhs[r] + Eb[r]), Eb[r]) * inv))) if nz else f32(0)
                thhi = min(thhi, f32(ratio + er))
            l1 = fma32(TT_HI, max(thhi, f32(1)), thhi)
            limhi = fma32(f32(4) * U, abs(l1), l1)
            exact_elig = [r for r in elig]
            best = min((rx[r] if rx[r] > Fraction(1, 10 ** 11) else Fraction(0)) / Tx[r][q] for r in exact_elig)
            lim_exact = best + Fraction(1, 10 ** 12) * max(best, 1)
            for r in amb:
                num = f32(rhs[r] - SAFE * Eb[r])
                lim = f32(limhi * f32(a[r] + SAFE * ea[r]))
                if not f32(num * f32(1 - 8 * U)) > lim:
                    return it
                STATS["uncertain_rows_passed"] += 1
                # were it eligible, its ratio could neither be the minimum
                # nor tie with it
                if Tx[r][q] > Fraction(1, 10 ** 9):
                    STATS["uncertain_rows_eligible"] += 1
                    check(rx[r] / Tx[r][q] > lim_exact)
        # the kernel's tie certification is exercised by the GPU parity tests;
        # here the exact minimum ratio row (unique in these samples) is taken
        # when the binary32 ratios separate it
        ratios = {}
        for r in elig:
            nz = rhs[r] > TS_HI + f32(1.25) * Eb[r]
            ratios[r] = Fraction(0) if not nz else rx[r] / Tx[r][q]
        best = min(ratios.values())
        tied = [r for r in elig if ratios[r] <= best + Fraction(1, 10 ** 12) * max(best, 1)]
        leave = min(tied, key=lambda r: basis[r])
        piv = a[leave]
        P = f32(f32(1) / piv)
        rho = f32(ea[leave] * P)
        if not rho <= 0.5:
            return it
        rr = fma32(f32(2) * rho, rho, rho)
        prow, Ep = [None] * K, [None] * K
        for k in range(K):
            pr = f32(T[leave][k] * P)
            eP = f32(E[leave][k] * P)
            prow[k] = f32(1) if k == q else pr
            Ep[k] = f32(0) if k == q else fma32(RCP_MUL, abs(pr), fma32(rr, f32(abs(pr) + eP), eP))
        prhs = f32(rhs[leave] * P)
        ebP = f32(Eb[leave] * P)
        Ebp = fma32(RCP_MUL, abs(prhs), fma32(rr, f32(abs(prhs) + ebP), ebP))
        for r in range(M):
            lr = r == leave
            ar = f32(-1) if lr else a[r]
            ear = f32(0) if lr else ea[r]
            aar = f32(abs(ar) + ear)
            for k in range(K):
                tn = fma32(-ar, prow[k], f32(0) if lr else T[r][k])
                en = fma32(U, abs(tn), fma32(aar, Ep[k], fma32(ear, abs(prow[k]), E[r][k])))
                T[r][k] = tn
                E[r][k] = Ep[k] if lr else en
            rn = fma32(-ar, prhs, f32(0) if lr else rhs[r])
            ebn = fma32(U, abs(rn), fma32(aar, Ebp, fma32(ear, abs(prhs), Eb[r])))
            rhs[r] = rn
            Eb[r] = Ebp if lr else ebn
        dq, edq = d[q], Ed[q]
        adq = f32(abs(dq) + edq)
        for k in range(K):
            d[k] = fma32(-dq, prow[k], d[k])
            Ed[k] = fma32(U, abs(d[k]), fma32(adq, Ep[k], fma32(edq, abs(prow[k]), Ed[k])))
        # the same pivot in exact arithmetic
        pivx = Tx[leave][q]
        prx = [Tx[leave][k] / pivx for k in range(K)]
        prhx = rx[leave] / pivx
        for r in range(M):
            if r == leave:
                continue
            arx = Tx[r][q]
            Tx[r] = [Tx[r][k] - arx * prx[k] for k in range(K)]
            rx[r] = rx[r] - arx * prhx
        Tx[leave] = prx
        rx[leave] = prhx
        dqx = dx_[q]
        dx_ = [dx_[k] - dqx * prx[k] for k in range(K)]
        lb = basis[leave]
        if lb >= M:
            basic[lb - M] = False
        else:
            n_art -= 1
        basic[q] = True
        basis[leave] = M + q
        it += 1
        sound()
    return it


def test_running_bounds_hold_and_certified_decisions_are_exact():
    rng = np.random.default_rng(20260)
    fails = []
    pivots = 0

    def check(ok):
        if not ok:
            fails.append(1)

    for _ in range(60):
        xi64, eta64, xs, es = columns(rng)
        pivots += run(xi64, eta64, xs, es, check)
    assert not fails, len(fails)
    assert pivots >= 150  # most samples pivot through phase I under certification


def test_uncertain_rows_passed_over_are_never_the_leaving_row():
    rng = np.random.default_rng(1508)
    fails = []

    def check(ok):
        if not ok:
            fails.append(1)

    STATS.update(uncertain_rows_passed=0, uncertain_rows_eligible=0)
    for _ in range(300):
        run(*lattice_columns(rng), check)
    # jittered neighbourhoods also give uncertain rows that are in fact
    # eligible (pivot elements just above 1e-9 under large bounds), where the
    # exact comparison with the tie limit has teeth
    rng = np.random.default_rng(5)
    for _ in range(600):
        run(*columns(rng), check)
    assert not fails, len(fails)
    assert STATS["uncertain_rows_passed"] > 0  # the rule is exercised
    assert STATS["uncertain_rows_eligible"] > 0


def test_a_planted_underestimate_is_caught():
    # the same replay with the conversion bounds of the offsets shrunk 1000
    # times: the entries leave their (too small) bounds at once
    global INIT
    keep = INIT
    INIT = f32(1e-3)
    try:
        rng = np.random.default_rng(20260)
        fails = []

        def check(ok):
            if not ok:
                fails.append(1)

        for _ in range(10):
            xi64, eta64, xs, es = columns(rng)
            run(xi64, eta64, xs, es, check)
        assert fails
    finally:
        INIT = keep
