"""The bound that lets a plan, and the pair lists built from it, be reused
across iterations (Sec. 5 sparsification at a fixed lengthscale): a pose that
passes the solver's drift test keeps every pair within the cutoff inside the
plan radius at the plan pose. The decisions are restated here in FP32 as the
solve kernel forms them (the drift test of an iteration's start, the plan-time
distance test of a pair list, the cluster-local cutoff test of a pass), on
pairs placed just inside the cutoff at poses whose drift is close to the
allowance. No GPU: this checks the margins of the argument, not the kernel."""
import numpy as np

F = np.float32


def fmaf(a, b, c):
    # a * b is exact in FP64 for FP32 operands; one rounding of the sum to
    # FP64 and one to FP32 (a fused FP32 FMA rounds once: the double rounding
    # can differ in the last bit, far below the margins tested here)
    return F(np.float64(a) * np.float64(b) + np.float64(c))


def transform(R, T, p):
    """R p + T in FP32 with the kernel's FMA chain (row r: R[r,0] x +
    (R[r,1] y + (R[r,2] z + T[r])))."""
    return np.array([fmaf(R[r, 0], p[0], fmaf(R[r, 1], p[1], fmaf(R[r, 2], p[2], T[r])))
                     for r in range(3)], dtype=F)


def rot(axis, ang):
    a = axis / np.linalg.norm(axis)
    K = np.array([[0, -a[2], a[1]], [a[2], 0, -a[0]], [-a[1], a[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def drift_ok(Rc, Tc, Rp, Tp, need, rp, src_radius_f):
    """The reuse test at an iteration's start: differences of the centred
    poses in FP64, the rest in FP32 with 2e-5 relative and 1e-6 r_c margins."""
    d = np.concatenate([(Rc - Rp).ravel(), Tc - Tp]).astype(F)
    sr = F(np.sum(d[:9] * d[:9], dtype=F))
    st = F(np.sum(d[9:] * d[9:], dtype=F))
    drift = F(fmaf(np.sqrt(sr), src_radius_f, np.sqrt(st)) * F(1 + 2e-5) + F(1e-6) * need)
    return bool(need + drift <= rp)


def pass_keeps(x, zt, o, rc2):
    """The pass's cutoff test relative to the staged cluster's origin o:
    t = x_l . (-2 z_l) + |z_l|^2 against r_c^2 - |x_l|^2."""
    zl = (zt - o).astype(F)
    m = np.array([F(-2) * zl[0], F(-2) * zl[1], F(-2) * zl[2],
                  fmaf(zl[0], zl[0], fmaf(zl[1], zl[1], F(zl[2] * zl[2])))], dtype=F)
    xl = (x - o).astype(F)
    x2 = fmaf(xl[0], xl[0], fmaf(xl[1], xl[1], F(xl[2] * xl[2])))
    t = fmaf(xl[0], m[0], fmaf(xl[1], m[1], fmaf(xl[2], m[2], m[3])))
    return bool(t <= F(rc2 - x2))


def listed(x, zp, rp2):
    d = (x - zp).astype(F)
    return bool(fmaf(d[0], d[0], fmaf(d[1], d[1], F(d[2] * d[2]))) <= rp2)


def _case(seed, ell, radius, drift_frac):
    rng = np.random.default_rng(seed)
    z = (rng.normal(size=(300, 3)) * radius / 2).clip(-radius, radius).astype(F)
    rc = np.sqrt(2 * ell * ell * np.log(1000.0))
    rc2 = F(rc * rc)
    need = F(np.sqrt(np.float64(rc2)) * 1.001)
    rp = F(np.float64(need) * 1.1)
    corner = np.abs(z).max(axis=0).astype(np.float64)
    src_radius_f = F(F(np.linalg.norm(corner)) * F(1 + 1e-6))
    Rp = rot(rng.normal(size=3), rng.uniform(0, np.pi))
    Tp = rng.normal(size=3) * 0.1
    # a move whose drift bound |dR|_F r_src + |dT| is drift_frac of the skin
    allow = float(rp - need)
    share = rng.uniform(0.2, 0.8)
    ang = share * drift_frac * allow / (np.sqrt(2.0) * float(src_radius_f))
    dR = rot(rng.normal(size=3), ang)
    dT = rng.normal(size=3)
    dT *= (1 - share) * drift_frac * allow / np.linalg.norm(dT)
    Rc, Tc = dR @ Rp, dR @ Tp + dT
    ok = drift_ok(Rc, Tc, Rp, Tp, need, rp, src_radius_f)
    Rpf, Tpf = Rp.astype(F), Tp.astype(F)
    Rcf, Tcf = Rc.astype(F), Tc.astype(F)
    kept = missed = 0
    for j in range(len(z)):
        zt = transform(Rcf, Tcf, z[j])
        zp = transform(Rpf, Tpf, z[j])
        # the cluster's origin: another staged point within about a cutoff radius
        o = (zt + rng.uniform(-rc, rc, size=3)).astype(F)
        for _ in range(8):
            u = rng.normal(size=3)
            x = (zt + u / np.linalg.norm(u) * rc * rng.uniform(0.97, 1.0)).astype(F)
            if pass_keeps(x, zt, o, rc2):
                kept += 1
                missed += 0 if listed(x, zp, F(rp * rp)) else 1
    return ok, kept, missed


def test_reused_plan_covers_the_kept_pairs():
    """Poses that pass the drift test, with the drift near the allowance:
    every pair the pass keeps was listed at the plan pose."""
    for seed, ell, radius in [(1, 0.02, 5.0), (2, 0.02, 30.0), (3, 0.05, 5.0), (4, 0.15, 3.0)]:
        ok, kept, missed = _case(seed, ell, radius, drift_frac=0.97)
        assert ok, (seed, "the move should pass the drift test")
        assert kept > 1000
        assert missed == 0, (seed, missed, kept)


def test_drift_beyond_the_skin_is_refused_and_would_miss_pairs():
    """The same construction with three times the allowed drift: the drift
    test refuses the pose, and a plan kept anyway would have missed pairs."""
    ok, kept, missed = _case(5, 0.02, 5.0, drift_frac=3.0)
    assert not ok
    assert missed > 0, kept
