"""The margin of the kernels' FP32 screen of the Section IV.D model.

The direct, tensor-core and FFT cores decide "model SNR >= target" first in
FP32 and fall back to the FP64 comparison only when the two sides are within
a relative margin of 2^-14, or when an operand or intermediate leaves
[1e-30, 1e30].  The claim is that the screen never decides differently from
the FP64 comparison.  This test restates the screen's operation sequence in
numpy float32 (IEEE single, one rounding per operation, as the device code
computes it without contraction; a fused multiply-add only rounds less) and
checks the claim on random operands and on operands placed on the threshold,
with the block moment perturbed by the largest error its FP32 conversion can
make.  The GPU test tests/test_gpu_selection_ties.py checks the kernels
themselves at the threshold."""
import numpy as np

f32, f64 = np.float32, np.float64
MARGIN = f32(1) + f32(2.0 ** -14)


def feasible64(s2s, Ms, s2k, Mk, S, K, thr):
    """The FP64 comparison, one correctly rounded operation at a time."""
    S2, K2 = f64(S) * f64(S), f64(K) * f64(K)
    Ms2, Mk2 = f64(Ms) * f64(Ms), f64(Mk) * f64(Mk)
    num = (f64(144.0) * (s2s * s2k)) * (S2 * K2)
    a = (s2s * S2) * Mk2
    c = (s2k * K2) * Ms2
    den = f64(12.0) * (a + c) + Ms2 * Mk2
    return num >= thr * den


def screen32(s2s, Ms, s2k, Mk, S, K, thr):
    with np.errstate(all="ignore"):
        S2, K2 = f32(S) * f32(S), f32(K) * f32(K)
        Ms2, Mk2 = Ms * Ms, Mk * Mk
        ss, SK = s2s * s2k, S2 * K2
        t144 = f32(144) * ss
        num = t144 * SK
        sa = s2s * S2
        a = sa * Mk2
        kc = s2k * K2
        c = kc * Ms2
        mm = Ms2 * Mk2
        den = f32(12) * (a + c) + mm
        rhs = thr * den
        vals = (s2s, s2k, Ms2, Mk2, ss, SK, t144, num, sa, a, kc, c, mm, den, rhs, thr)
        if not all(np.isfinite(v) and f32(1e-30) <= v <= f32(1e30) for v in vals):
            return 0
        if num >= rhs * MARGIN:
            return 1
        if num * MARGIN <= rhs:
            return -1
        return 0


def test_screen_never_contradicts_fp64():
    rng = np.random.default_rng(20130118)
    decided = 0
    for it in range(20000):
        Ms, Mk = f32(10 ** rng.uniform(-8, 8)), f32(10 ** rng.uniform(-8, 8))
        s2s = f64(Ms) ** 2 * 10 ** rng.uniform(-6, 0)
        s2k = f64(Mk) ** 2 * 10 ** rng.uniform(-6, 0)
        S, K = int(rng.integers(1, 2049)), int(rng.integers(1, 2049))
        if it % 2:  # on the threshold, to within a few parts in 10^4
            S2, K2 = f64(S) ** 2, f64(K) ** 2
            num = 144 * s2s * s2k * S2 * K2
            den = 12 * (s2s * S2 * f64(Mk) ** 2 + s2k * K2 * f64(Ms) ** 2) + f64(Ms) ** 2 * f64(Mk) ** 2
            thr = num / den * (1 + rng.uniform(-3e-4, 3e-4))
        else:
            thr = 10 ** rng.uniform(0, 8)
        # the block moment reaches the screen through a split 64-bit -> FP32
        # conversion and one division: within 2^-22 relative
        s2s_f = f32(f32(s2s) * f32(1 + rng.uniform(-2.0 ** -22, 2.0 ** -22)))
        sc = screen32(s2s_f, Ms, f32(s2k), Mk, S, K, f32(thr))
        if sc:
            decided += 1
            assert (sc > 0) == feasible64(s2s, Ms, s2k, Mk, S, K, thr), (it, sc)
    assert decided > 12000  # the screen decides most random operands


def test_screen_leaves_exact_ties_open():
    """A threshold equal to the model value (to FP64 rounding) is never
    decided in FP32."""
    rng = np.random.default_rng(7)
    for _ in range(2000):
        Ms, Mk = f32(rng.uniform(0.1, 10)), f32(rng.uniform(0.1, 10))
        s2s, s2k = f64(Ms) ** 2 * rng.uniform(0.01, 1), f64(Mk) ** 2 * rng.uniform(0.01, 1)
        S, K = int(rng.integers(2, 2049)), int(rng.integers(2, 2049))
        S2, K2 = f64(S) ** 2, f64(K) ** 2
        thr = (144 * s2s * s2k * S2 * K2) / (12 * (s2s * S2 * f64(Mk) ** 2 + s2k * K2 * f64(Ms) ** 2)
                                            + f64(Ms) ** 2 * f64(Mk) ** 2)
        assert screen32(f32(s2s), Ms, f32(s2k), Mk, S, K, f32(thr)) == 0
