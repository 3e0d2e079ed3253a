"""Pins for the FP64 oracle: each test checks it against something other than itself.

* the matrices the paper prints (golden fixtures under tests/golden/);
* the Appendix listing, restated with ``scipy.signal.convolve2d`` (a library 2-D convolution
  with MATLAB's conv2 'same' semantics) and numpy's first-index argmin;
* closed forms derived by hand from the Sec. IV-B kernels (affine ramps, the paraboloid x^2,
  impulses, step edges, a square);
* exact invariants (contrast, D4 symmetry, the max principle of the explicit update);
* a scalar recursion worked by hand for the primal-dual update of Sec. V-C;
* numpy's float16 rounding for the storage emulation.
"""
from fractions import Fraction
import os

import numpy as np
import pytest
from scipy.signal import convolve2d, correlate2d

import oracle
from paper_1903_07189_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_blocks(name):
    """Parse a golden kernel file into {name: (rows of Fractions, denominator)}."""
    blocks, cur, rows, den = {}, None, [], 1
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            if line.startswith("/"):
                den = int(line[1:])
                continue
            parts = line.split()
            if len(parts) == 1 and not parts[0].lstrip("-").replace("/", "").isdigit():
                if cur is not None:
                    blocks[cur] = (rows, den)
                cur, rows, den = parts[0], [], 1
            else:
                rows.append([Fraction(p) for p in parts])
    blocks[cur] = (rows, den)
    return {k: np.array([[float(v) / d for v in r] for r in rows]) for k, (rows, d) in blocks.items()}


PRINTED = _read_blocks("kernels_h1_h8.txt")
APPENDIX = _read_blocks("appendix_k1_k2.txt")
K4 = _read_blocks("laplace_k4.txt")["k4"]


# ---------------------------------------------------------------- kernel table (Sec. IV-B)
def test_printed_kernels_shape():
    """Each printed h_i: centre -1, off-centre weights >= 0 summing to 1, six taps (Sec. IV-D)."""
    for i in range(1, 9):
        k = PRINTED[f"h{i}"]
        assert k[1, 1] == -1.0
        off = k.copy()
        off[1, 1] = 0
        assert (off >= 0).all()
        assert abs(off.sum() - 1.0) < 1e-15
        assert np.count_nonzero(k) == 6


def test_oracle_kernel_table_is_the_printed_one():
    for i in range(8):
        np.testing.assert_allclose(oracle.kernel(i), PRINTED[f"h{i + 1}"], rtol=0, atol=1e-16)


def test_antipodal_kernels_average_to_k4():
    """h1+h3 = h2+h4 = h5+h7 = h6+h8 = 2*k4 (k4 of Eq. kernel3)."""
    for a, b in [(1, 3), (2, 4), (5, 7), (6, 8)]:
        np.testing.assert_allclose(PRINTED[f"h{a}"] + PRINTED[f"h{b}"], 2 * K4, atol=1e-15)
        np.testing.assert_allclose(oracle.kernel(a - 1) + oracle.kernel(b - 1), 2 * K4, atol=1e-15)


# ------------------------------------------------- the Appendix listing, via scipy's conv2
def _appendix_wmc(u, boundary):
    """Restatement of the Appendix function with a library convolution.

    The kernels are scaled to integers (x12) so that integer images are evaluated exactly;
    the listing's order of the eight convolutions and its first-minimum rule are kept.
    """
    k1 = APPENDIX["k1"] * 12
    k2 = APPENDIX["k2"] * 12
    ks = [k1, np.fliplr(k1), k1.T, np.flipud(k1.T), k2, np.fliplr(k2), np.flipud(k2), np.rot90(k2, 2)]
    if boundary == "zero":
        dist = np.stack([convolve2d(u, k, mode="same", boundary="fill", fillvalue=0) for k in ks], -1)
    else:
        up = np.pad(u, 1, mode="edge")
        dist = np.stack([convolve2d(up, k, mode="valid") for k in ks], -1)
    ind = np.argmin(np.abs(dist), axis=-1)  # first minimum, like MATLAB's min
    return np.take_along_axis(dist, ind[..., None], -1)[..., 0] / 12.0, dist / 12.0


@pytest.mark.parametrize("boundary", ["zero", "replicate"])
@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (6, 1), (2, 2), (5, 5), (13, 17), (32, 24)])
def test_matches_appendix_on_integer_images(boundary, shape):
    """Integer images: both sides are exact, so values and tie choices must agree bit for bit."""
    rng = np.random.default_rng(hash(shape) % 2**32)
    for trial in range(4):
        hi = [2, 5, 50, 1000][trial]
        u = rng.integers(-hi, hi + 1, size=shape).astype(np.float64)
        want, _ = _appendix_wmc(u, boundary)
        got = oracle.wmc_eval(u, boundary)
        assert np.array_equal(got, want), (boundary, shape, hi)


@pytest.mark.parametrize("boundary", ["zero", "replicate"])
def test_matches_appendix_on_real_images(boundary):
    """Real-valued images: same candidate sets; the same value wherever the minimum is clear."""
    u = synth.make_image(40, 56, seed=7, sigma=0.05).astype(np.float64)
    want, dist = _appendix_wmc(u, boundary)
    got, cand, _ = oracle.wmc_eval(u, boundary, candidates=True)
    np.testing.assert_allclose(np.sort(cand, -1), np.sort(dist, -1), rtol=0, atol=1e-14)
    mags = np.sort(np.abs(dist), -1)
    clear = (mags[..., 1] - mags[..., 0]) > 1e-12
    assert clear.mean() > 0.99
    np.testing.assert_allclose(got[clear], want[clear], rtol=0, atol=1e-14)


# ------------------------------------------------------------- closed forms, derived by hand
def test_affine_candidates_closed_form():
    """U = a x + b y + c (x = column, y = row): interior d_1..d_8 =
    -2a/3, -2b/3, 2a/3, 2b/3, -(a+b)/2, (a-b)/2, (a+b)/2, -(a-b)/2."""
    rng = np.random.default_rng(1)
    y, x = np.mgrid[0:9, 0:11].astype(np.float64)
    for _ in range(20):
        a, b, c = rng.normal(size=3)
        u = a * x + b * y + c
        _, cand, _ = oracle.wmc_eval(u, "replicate", candidates=True)
        want = np.array([-2 * a / 3, -2 * b / 3, 2 * a / 3, 2 * b / 3,
                         -(a + b) / 2, (a - b) / 2, (a + b) / 2, -(a - b) / 2])
        np.testing.assert_allclose(cand[1:-1, 1:-1], np.broadcast_to(want, cand[1:-1, 1:-1].shape),
                                   rtol=0, atol=1e-12)


def test_affine_magnitude_and_zero_directions():
    """|H^w| = min(2|a|/3, 2|b|/3, |a+b|/2, |a-b|/2); zero exactly along the 8 normals."""
    y, x = np.mgrid[0:7, 0:7].astype(np.float64)
    for a, b in [(3, 0), (0, -5), (2, 2), (4, -4), (3, 1), (-2, 7), (1, 2)]:
        u = a * x + b * y + 0.25
        hw = oracle.wmc_eval(u, "replicate")[1:-1, 1:-1]
        mag = min(2 * abs(a) / 3, 2 * abs(b) / 3, abs(a + b) / 2, abs(a - b) / 2)
        np.testing.assert_allclose(np.abs(hw), mag, rtol=0, atol=1e-12)
        if a == 0 or b == 0 or abs(a) == abs(b):
            assert np.all(hw == 0)


def test_ramp_canonical_tie_choice():
    """U = x + 2y: candidates +-2/3, +-4/3, +-3/2, +-1/2 in the interior.  The minimum |d| = 1/2
    is shared by d_6 = -1/2 and d_8 = +1/2 (an opposite-sign tie).  The Appendix's list, read as
    correlation kernels, is (h3, h1, h4, h2, h7, h8, h6, h5): h8 comes before h6, so its first
    minimum is d_8 = +1/2."""
    y, x = np.mgrid[0:5, 0:5].astype(np.float64)
    hw, cand, idx = oracle.wmc_eval(x + 2 * y, "replicate", candidates=True)
    assert np.all(hw[1:-1, 1:-1] == 0.5)
    assert np.all(idx[1:-1, 1:-1] == 8)


def test_paraboloid_x2():
    """U = x^2: d_2 = d_4 = 2/3 everywhere inside; d_1 = 2/3 - 4x/3, d_3 = 2/3 + 4x/3,
    d_5 = d_8 = 2/3 - x, d_6 = d_7 = 2/3 + x."""
    y, x = np.mgrid[0:8, 0:9].astype(np.float64)
    _, cand, _ = oracle.wmc_eval(x ** 2, "replicate", candidates=True)
    xi = x[1:-1, 1:-1]
    want = np.stack([2 / 3 - 4 * xi / 3, 2 / 3 + 0 * xi, 2 / 3 + 4 * xi / 3, 2 / 3 + 0 * xi,
                     2 / 3 - xi, 2 / 3 + xi, 2 / 3 + xi, 2 / 3 - xi], -1)
    np.testing.assert_allclose(cand[1:-1, 1:-1], want, rtol=0, atol=1e-12)


def test_paraboloid_vertex():
    """U = (x-3)^2 + (y-3)^2: every d_i = 4/3 at the vertex."""
    y, x = np.mgrid[0:7, 0:7].astype(np.float64)
    _, cand, _ = oracle.wmc_eval((x - 3) ** 2 + (y - 3) ** 2, "replicate", candidates=True)
    np.testing.assert_allclose(cand[3, 3], np.full(8, 4 / 3), rtol=0, atol=1e-14)


@pytest.mark.parametrize("boundary", ["replicate", "zero"])
def test_impulse(boundary):
    """A unit impulse: -1 at the impulse (all d_i = -1), 0 at every other pixel (some half
    window avoids it)."""
    u = np.zeros((7, 8))
    u[3, 4] = 1
    hw = oracle.wmc_eval(u, boundary)
    want = np.zeros_like(u)
    want[3, 4] = -1
    assert np.array_equal(hw, want)


def test_step_edges_vanish():
    """Axis-aligned steps vanish everywhere (replicate keeps them steps); diagonal steps vanish
    at interior pixels: the half window on one side of the edge sees a constant."""
    y, x = np.mgrid[0:12, 0:13].astype(np.float64)
    for u in [(x >= 5) * 1.0, (y >= 4) * 2.0, (x < 7) * -3.0]:
        assert np.all(oracle.wmc_eval(u, "replicate") == 0)
    for u in [(x + y >= 9) * 1.0, (x - y >= 2) * 1.5, (x + y < 12) * 1.0]:
        assert np.all(oracle.wmc_eval(u, "replicate")[1:-1, 1:-1] == 0)


def test_square_corners():
    """A 3x3 square of ones in a 5x5 zero image: -1/6 at its four corners (h7 or a rotation
    of it sees 1/6 + 2/3 + 0 - 1), 0 everywhere else."""
    u = np.zeros((5, 5))
    u[1:4, 1:4] = 1
    hw = oracle.wmc_eval(u, "replicate")
    want = np.zeros((5, 5))
    for yy, xx in [(1, 1), (1, 3), (3, 1), (3, 3)]:
        want[yy, xx] = -1 / 6
    np.testing.assert_allclose(hw, want, rtol=0, atol=1e-15)


def test_constant_image():
    for bnd in ["replicate", "zero"]:
        hw = oracle.wmc_eval(np.full((4, 6), 2.5), bnd)
        if bnd == "replicate":
            assert np.all(hw == 0)
        else:
            assert np.all(hw[1:-1, 1:-1] == 0)


# --------------------------------------------------------------------------- invariances
def test_contrast_homogeneity_bitwise():
    """H^w(alpha U) = alpha H^w(U) bit for bit when alpha is +-2^k (Sec. III-B, exact here)."""
    u = synth.make_image(33, 29, seed=3).astype(np.float64)
    hw = oracle.wmc_eval(u)
    for alpha in [2.0, -2.0, 0.5, -0.25, 1024.0, -1.0]:
        assert np.array_equal(oracle.wmc_eval(alpha * u), alpha * hw)


def test_contrast_homogeneity_general():
    u = synth.make_image(33, 29, seed=3).astype(np.float64)
    hw, cand, _ = oracle.wmc_eval(u, candidates=True)
    mags = np.sort(np.abs(cand), -1)
    clear = (mags[..., 1] - mags[..., 0]) > 1e-9
    for alpha in [3.7, -0.3]:
        np.testing.assert_allclose(oracle.wmc_eval(alpha * u)[clear], alpha * hw[clear], rtol=1e-12,
                                   atol=1e-14)


def test_offset_invariance():
    u = synth.make_image(20, 20, seed=4).astype(np.float64)
    np.testing.assert_allclose(oracle.wmc_eval(u + 3.0), oracle.wmc_eval(u), atol=1e-13)
    ui = np.random.default_rng(0).integers(0, 9, (9, 9)).astype(np.float64)
    assert np.array_equal(oracle.wmc_eval(ui + 7), oracle.wmc_eval(ui))


@pytest.mark.parametrize("op", ["rot90", "rot180", "rot270", "fliplr", "flipud", "transpose"])
def test_d4_equivariance_off_ties(op):
    """The kernel set is closed under the dihedral group, so H^w(R U) = R H^w(U) wherever the
    minimum |d_i| is unique (Sec. IV-A: eight normals 45 degrees apart)."""
    f = {"rot90": lambda a: np.rot90(a, 1), "rot180": lambda a: np.rot90(a, 2),
         "rot270": lambda a: np.rot90(a, 3), "fliplr": np.fliplr, "flipud": np.flipud,
         "transpose": lambda a: a.T}[op]
    u = synth.make_image(24, 31, seed=5).astype(np.float64)
    hw, cand, _ = oracle.wmc_eval(u, candidates=True)
    mags = np.sort(np.abs(cand), -1)
    clear = f((mags[..., 1] - mags[..., 0]) > 1e-9)
    got = oracle.wmc_eval(np.ascontiguousarray(f(u)))
    np.testing.assert_allclose(got[clear], f(hw)[clear], rtol=0, atol=1e-13)


# --------------------------------------------------------------------- flows (Sec. V-B, MCF)
def test_max_principle():
    """With step*(1+lambda) <= 1 every step is a convex combination of neighbours and f, so all
    iterates stay inside [min f, max f]."""
    f = synth.make_image(30, 30, seed=6, sigma=0.1).astype(np.float64)
    lo, hi = f.min(), f.max()
    for lam, step in [(1.0, 0.5), (1.0, 0.25), (2.0, 1 / 3), (0.5, 0.5)]:
        for it in [1, 5, 40]:
            u = oracle.denoise(f, lam, step, it)
            assert u.min() >= lo - 1e-12 and u.max() <= hi + 1e-12


def test_one_step_by_hand():
    """One step, lambda = 1, step = 1/4, on a 3x3 image with a single 1 in the middle:
    H^w = -1 there and 0 elsewhere, so U^1 = f + (1/4)(H^w - (f - f)) = f + H^w/4."""
    f = np.zeros((3, 3))
    f[1, 1] = 1
    u1 = oracle.denoise(f, 1.0, 0.25, 1)
    want = f.copy()
    want[1, 1] = 0.75
    np.testing.assert_allclose(u1, want, atol=1e-16)


def test_two_steps_by_hand():
    """Second step of the same problem: now U = 0.75 at the centre, f = 1 there.  The centre's
    d_i are all -0.75; every neighbour still has a half window that avoids the centre, so
    U^2 = U^1 + (1/4)(-0.75 - (0.75 - 1)) at the centre = 0.75 - 0.125 = 0.625."""
    f = np.zeros((3, 3))
    f[1, 1] = 1
    u2 = oracle.denoise(f, 1.0, 0.25, 2)
    want = np.zeros((3, 3))
    want[1, 1] = 0.625
    np.testing.assert_allclose(u2, want, atol=1e-16)


def test_denoise_contrast_bitwise():
    f = synth.make_image(26, 19, seed=8).astype(np.float64)
    u = oracle.denoise(f, 1.0, 0.25, 10)
    for alpha in [2.0, -0.5]:
        assert np.array_equal(oracle.denoise(alpha * f, 1.0, 0.25, 10), alpha * u)


def test_resume():
    """denoise(f, n + m) == m more steps from U^n, bit for bit (the state is (U, f))."""
    f = synth.make_image(21, 23, seed=9).astype(np.float64)
    un = oracle.denoise(f, 1.2, 0.2, 7)
    assert np.array_equal(oracle.denoise(f, 1.2, 0.2, 12), oracle.denoise(f, 1.2, 0.2, 5, u0=un))


def test_mcf_fixed_points():
    y, x = np.mgrid[0:9, 0:10].astype(np.float64)
    for u in [np.full((9, 10), 0.3), (x >= 4) * 1.0, (y >= 6) * 1.0]:
        assert np.array_equal(oracle.mcf(u, 0.5, 20), u)


def test_mcf_is_flow_without_data_term():
    u = synth.make_image(15, 15, seed=10).astype(np.float64)
    hw = oracle.wmc_eval(u)
    np.testing.assert_allclose(oracle.mcf(u, 0.3, 1), u + 0.3 * hw, atol=1e-16)


def test_energies():
    y, x = np.mgrid[0:8, 0:8].astype(np.float64)
    step = (x >= 3) * 1.0
    e = oracle.energies(step, step, step)
    assert e == (0.0, 0.0, 0.0)
    imp = np.zeros((6, 6))
    imp[2, 3] = 2.0
    e = oracle.energies(imp, np.zeros((6, 6)), np.ones((6, 6)))
    assert e[0] == pytest.approx(2.0, abs=1e-15)       # only the impulse: |H^w| = 2
    assert e[1] == pytest.approx(0.5 * 4.0, abs=1e-15)  # 1/2 * 2^2
    assert e[2] == pytest.approx(35 * 1.0 + 1.0, abs=1e-15)


# ------------------------------------------------------------------ primal-dual (Sec. V-C)
def test_primal_dual_scalar_by_hand():
    """lambda = 0 (no regulariser): the update is pointwise.  f = 0, U^0 = 1, alpha = 0.5,
    step = 0.1:  r = 1 -> d^1 = 0.5, U^1 = 1 - 0.1 (1 - 0)/0.5 = 0.8;
    r = 0.8 + 0.5 = 1.3 -> d^2 = 0.5, U^2 = 0.8 - 0.1 (1 - 0.5)/0.5 = 0.7."""
    f = np.zeros((3, 4))
    u0 = np.ones((3, 4))
    u1, d1 = oracle.l1_primal_dual(f, 0.0, 0.1, 0.5, 1, u0=u0)
    np.testing.assert_allclose(u1, 0.8, atol=1e-15)
    np.testing.assert_allclose(d1, 0.5, atol=1e-15)
    u2, d2 = oracle.l1_primal_dual(f, 0.0, 0.1, 0.5, 2, u0=u0)
    np.testing.assert_allclose(u2, 0.7, atol=1e-15)
    np.testing.assert_allclose(d2, 0.5, atol=1e-15)


def test_primal_dual_inside_clip():
    """|r| <= alpha throughout: d^{t+1} = r.  f = 0, U^0 = 0.1, alpha = 1, step = 0.1, lambda = 0:
    d^1 = 0.1, U^1 = 0.1 - 0.1 * 0.2 = 0.08;  d^2 = 0.08 + 0.1 = 0.18,
    U^2 = 0.08 - 0.1 * (0.36 - 0.1) = 0.054."""
    f = np.zeros((2, 2))
    u2, d2 = oracle.l1_primal_dual(f, 0.0, 0.1, 1.0, 2, u0=np.full((2, 2), 0.1))
    np.testing.assert_allclose(u2, 0.054, atol=1e-15)
    np.testing.assert_allclose(d2, 0.18, atol=1e-15)


def test_primal_dual_constant_is_fixed():
    f = np.full((5, 6), 0.4)
    u, d = oracle.l1_primal_dual(f, 2.0, 0.1, 0.3, 10)
    np.testing.assert_allclose(u, f, atol=1e-16)
    assert np.all(d == 0)


def test_primal_dual_resume_is_exact():
    """(U^n, d^n) carry the whole state: n + m iterations equal n, then m from (U^n, d^n)."""
    f = synth.make_image(21, 17, seed=41, sigma=0.1, dtype=np.float64)
    u7, d7 = oracle.l1_primal_dual(f, 1.5, 0.05, 0.08, 7)
    u3, d3 = oracle.l1_primal_dual(f, 1.5, 0.05, 0.08, 3)
    u7b, d7b = oracle.l1_primal_dual(f, 1.5, 0.05, 0.08, 4, u0=u3, d0=d3)
    assert np.array_equal(u7, u7b) and np.array_equal(d7, d7b)


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_primal_dual_large_alpha_is_curvature_flow(bnd):
    """alpha -> infinity: d stays tiny relative to alpha, the data term (2d^{t+1} - d^t)/alpha
    vanishes, and one iteration is one mean-curvature-flow step U + step*lambda*H^w(U)
    (Eq. MCF), which pins how lambda and H^w enter the update."""
    f = synth.make_image(19, 23, seed=42, sigma=0.1, dtype=np.float64)
    u0 = f + 0.3 * synth.make_image(19, 23, seed=43, sigma=0.05, dtype=np.float64)
    u1, _ = oracle.l1_primal_dual(f, 1.7, 0.2, 1e12, 1, bnd, u0=u0)
    np.testing.assert_allclose(u1, oracle.mcf(u0, 0.2 * 1.7, 1, bnd), rtol=0, atol=1e-10)


# ------------------------------------------------------------------- storage emulation
def test_round_f16_matches_numpy():
    rng = np.random.default_rng(11)
    vals = np.concatenate([rng.normal(size=2000), rng.normal(size=200) * 1e-6,
                           rng.normal(size=200) * 3e4, [6.1e-5, 5.96e-8, 2.98e-8, 65519.0, 65520.0, 1.0],
                           1 + (2 * np.arange(50) + 1) * 2.0 ** -11])
    np.testing.assert_array_equal(oracle.round_storage(vals, "f16"),
                                  vals.astype(np.float16).astype(np.float64))


def test_round_bf16_ties_and_carries():
    # bf16 keeps 8 significant bits: 1 + k/128 are representable; halfway points go to even.
    assert oracle.round_storage(np.array([1 + 1 / 256]), "bf16")[0] == 1.0
    assert oracle.round_storage(np.array([1 + 3 / 256]), "bf16")[0] == 1 + 4 / 256
    assert oracle.round_storage(np.array([1 + 1 / 256 + 1e-12]), "bf16")[0] == 1 + 1 / 128
    assert oracle.round_storage(np.array([255.5 * 2 ** -7 * 2]), "bf16")[0] == 4.0
    assert oracle.round_storage(np.array([-0.3]), "bf16")[0] == -0.30078125


def test_round_f32_matches_cast():
    vals = np.random.default_rng(12).normal(size=1000)
    np.testing.assert_array_equal(oracle.round_storage(vals, "f32"), vals.astype(np.float32).astype(np.float64))


# ------------------------------------------------------ unrolled denoising and its gradient
def test_unrolled_grad_lambda_zero_closed_form():
    """lambda = 0: U^t = f for every t, so loss = mean((f - clean)^2), dloss/df = 2 (f - clean)/N
    and dloss/dlambda = step sum_t (1-step)^(K-1-t) sum_p g^K H^w(f) = (1 - (1-step)^K) sum_p g^K H^w(f)."""
    f, clean = synth.make_image(12, 15, seed=40, sigma=0.1, return_clean=True)
    f, clean = f.astype(np.float64), clean.astype(np.float64)
    step, K = 0.3, 9
    loss, dl, df = oracle.unrolled_grad(f, clean, 0.0, step, K)
    gK = 2 * (f - clean) / f.size
    assert loss == pytest.approx(np.mean((f - clean) ** 2), rel=1e-14)
    np.testing.assert_allclose(df, gK, rtol=0, atol=1e-15)
    want = (1 - (1 - step) ** K) * np.sum(gK * oracle.wmc_eval(f))
    assert dl == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_unrolled_grad_matches_finite_differences(bnd):
    """Central differences of the plain forward (oracle.denoise, a separate code path) against
    the chain-rule gradient, for lambda and for f at a few pixels (steps too small to switch a
    selection)."""
    f, clean = synth.make_image(10, 13, seed=41, sigma=0.1, return_clean=True)
    f, clean = f.astype(np.float64), clean.astype(np.float64)
    lam, step, K = 1.3, 0.2, 7
    loss, dl, df = oracle.unrolled_grad(f, clean, lam, step, K, bnd)
    assert loss == pytest.approx(oracle.unrolled_loss(f, clean, lam, step, K, bnd), rel=1e-13)
    eps = 1e-6
    fd = (oracle.unrolled_loss(f, clean, lam + eps, step, K, bnd)
          - oracle.unrolled_loss(f, clean, lam - eps, step, K, bnd)) / (2 * eps)
    assert dl == pytest.approx(fd, rel=1e-6, abs=1e-12)
    for (y, x) in [(0, 0), (4, 6), (9, 12), (5, 0), (0, 7)]:
        fp, fm = f.copy(), f.copy()
        fp[y, x] += eps
        fm[y, x] -= eps
        fdf = (oracle.unrolled_loss(fp, clean, lam, step, K, bnd)
               - oracle.unrolled_loss(fm, clean, lam, step, K, bnd)) / (2 * eps)
        assert df[y, x] == pytest.approx(fdf, rel=1e-5, abs=1e-11), (y, x)


def test_unrolled_grad_zero_steps():
    f, clean = synth.make_image(6, 7, seed=42, return_clean=True)
    loss, dl, df = oracle.unrolled_grad(f, clean, 1.0, 0.25, 0)
    assert dl == 0.0
    np.testing.assert_allclose(df, 2 * (f.astype(np.float64) - clean) / f.size, atol=1e-16)


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_energy_grad_matches_finite_differences(bnd):
    u = synth.make_image(9, 11, seed=43, sigma=0.1).astype(np.float64)
    g = oracle.energy_grad(u, bnd)
    eps = 1e-7
    for (y, x) in [(0, 0), (4, 5), (8, 10), (0, 5), (3, 0)]:
        up, um = u.copy(), u.copy()
        up[y, x] += eps
        um[y, x] -= eps
        fd = (oracle.energies(up, boundary=bnd)[0] - oracle.energies(um, boundary=bnd)[0]) / (2 * eps)
        assert g[y, x] == pytest.approx(fd, rel=1e-5, abs=1e-8), (y, x)


def test_energy_grad_impulse_by_hand():
    """A unit impulse: only the impulse pixel has H^w != 0 (-1, every kernel); its selected
    kernel is h3 (first in the Appendix order), so dE/dU = -h3 centred on the impulse:
    +1 at the centre, -1/6 at N, NE, S, SE and -1/3 at E."""
    u = np.zeros((5, 5))
    u[2, 2] = 1
    g = oracle.energy_grad(u)
    want = np.zeros((5, 5))
    want[2, 2] = 1.0
    for (y, x) in [(1, 2), (1, 3), (3, 2), (3, 3)]:
        want[y, x] = -1 / 6
    want[2, 3] = -1 / 3
    np.testing.assert_allclose(g, want, atol=1e-15)


# ------------------------------------------- conventional finite-difference WMC (Eq. rhs)
def _grid(h, w):
    y, x = np.mgrid[0:h, 0:w].astype(np.float64)
    return y, x


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_fd_straight_level_lines_give_zero(bnd):
    """U depending on x alone has straight level lines: curvature 0 at every interior pixel
    (and, under REPLICATE, at the border too)."""
    y, x = _grid(12, 17)
    u = np.sin(0.4 * x) + 0.1 * x * x
    hw = oracle.fd_eval(u, bnd)
    inner = hw[1:-1, 1:-1] if bnd == "zero" else hw
    np.testing.assert_allclose(inner, 0.0, atol=1e-12)


def test_fd_paraboloid_is_two():
    """U = (x-cx)^2 + (y-cy)^2: central differences are exact on quadratics, grad = 2(x-cx, y-cy),
    Laplacian 4, normal second derivative 2, so H = 2 wherever the gradient is non-zero; the
    centre (zero gradient) gives 0 by definition."""
    y, x = _grid(11, 13)
    u = (x - 6.0) ** 2 + (y - 5.0) ** 2
    hw = oracle.fd_eval(u, "replicate")
    expect = np.full(u.shape, 2.0)
    expect[5, 6] = 0.0
    np.testing.assert_allclose(hw[1:-1, 1:-1], expect[1:-1, 1:-1], atol=1e-12)


def test_fd_saddle_closed_form():
    """U = (x-a)(y-b): U_x = y-b, U_y = x-a, U_xy = 1, U_xx = U_yy = 0, so
    H = -2 (x-a)(y-b) / ((x-a)^2 + (y-b)^2)."""
    y, x = _grid(9, 10)
    X, Y = x - 4.5, y - 3.5
    hw = oracle.fd_eval(X * Y, "replicate")
    expect = -2.0 * X * Y / (X * X + Y * Y)
    np.testing.assert_allclose(hw[1:-1, 1:-1], expect[1:-1, 1:-1], atol=1e-12)


def test_fd_gaussian_matches_continuous_wmc():
    """A radial Gaussian g(r) = exp(-r^2 / (2 s^2)) has circular level lines; Eq. wmc gives
    |grad U| * div(grad U / |grad U|) = g'(r) / r = -g / s^2.  Central differences converge to it
    at second order in 1/s."""
    s = 12.0
    y, x = _grid(81, 81)
    r2 = (x - 40.0) ** 2 + (y - 40.0) ** 2
    g = np.exp(-r2 / (2 * s * s))
    hw = oracle.fd_eval(g, "replicate")
    cont = -g / (s * s)
    sel = (r2 > 4.0) & (r2 < (2.5 * s) ** 2)
    rel = np.abs(hw[sel] - cont[sel]).max() / np.abs(cont[sel]).max()
    assert rel < 0.02, rel


@pytest.mark.parametrize("bnd", ["replicate", "zero"])
def test_fd_rotation_and_flip_equivariance(bnd):
    u = synth.make_image(15, 15, seed=61, sigma=0.1, dtype=np.float64)
    hw = oracle.fd_eval(u, bnd)
    np.testing.assert_allclose(oracle.fd_eval(np.rot90(u).copy(), bnd), np.rot90(hw), atol=1e-12)
    np.testing.assert_allclose(oracle.fd_eval(u[:, ::-1].copy(), bnd), hw[:, ::-1], atol=1e-12)
    np.testing.assert_allclose(oracle.fd_eval(u.T.copy(), bnd), hw.T, atol=1e-12)


def test_fd_flow_without_regulariser_relaxes_to_f():
    """lambda = 0: U^t = f + (1 - step)^t (U^0 - f) exactly (pins mu, the sign of the data term
    and the step count)."""
    f = synth.make_image(8, 9, seed=62, sigma=0.1, dtype=np.float64)
    u0 = f + 0.25
    out = oracle.fd_flow(f, 0.0, 0.3, 5, u0=u0)
    np.testing.assert_allclose(out, f + 0.7 ** 5 * 0.25, atol=1e-14)


def test_fd_flow_one_step_uses_fd_operator():
    """One mean-curvature step (f None) is U + step * lambda * H_fd(U)."""
    u = synth.make_image(10, 12, seed=63, sigma=0.1, dtype=np.float64)
    out = oracle.fd_flow(None, 2.0, 0.1, 1, mu=0.0, u0=u)
    np.testing.assert_allclose(out, u + 0.2 * oracle.fd_eval(u), atol=1e-14)


# ------------------------------------------------------------- worked 5x5 examples
def test_ramp_zero_boundary_rows_by_hand():
    """U = x + 2y on 5x5 with the Appendix's zero padding.  At (0,0) the only in-image
    neighbours are E = 1, S = 2, SE = 3, and the north-west half window h5 (2nw + 4n + ne + 4w -
    12c + sw)/12 reads none of them: d5 = 0, so H^w = 0.  The other entries follow the same way
    (exact rationals from the eight printed kernels, ties by the canonical order)."""
    y, x = np.mgrid[0:5, 0:5].astype(np.float64)
    hw = oracle.wmc_eval(x + 2 * y, "zero")
    np.testing.assert_allclose(hw[0], [0, 0, 1 / 2, 1 / 6, -1 / 6], atol=1e-15)
    np.testing.assert_allclose(hw[4], [-11 / 6, -4 / 3, -4 / 3, -4 / 3, -7 / 2], atol=1e-15)
    hr = oracle.wmc_eval(x + 2 * y, "replicate")
    assert abs(hr[0, 0] - 1 / 4) < 1e-15 and abs(hr[4, 4] + 1 / 4) < 1e-15


def test_one_step_on_a_mod7_image_by_hand():
    """One denoising step, lambda = 1, step = 1/4, REPLICATE, f[y][x] = ((3x + 5y) mod 7) / 7,
    U^0 = f, so U^1 = f + H^w(f)/4; the values were worked out in exact rationals."""
    y, x = np.mgrid[0:5, 0:5].astype(np.float64)
    f = ((3 * x + 5 * y) % 7) / 7
    u1 = oracle.denoise(f, 1.0, 0.25, 1)
    for (r, c), want in [((0, 0), 1 / 42), ((1, 1), 11 / 48), ((2, 2), 17 / 56), ((4, 4), 191 / 336)]:
        assert abs(u1[r, c] - want) < 1e-15, (r, c, u1[r, c], want)


# ------------------------------------------------- scale behaviour on smooth shapes
def smooth_disk(R, wf=0.25, margin=3.0):
    """U = (1 + tanh((R - r) / (wf R))) / 2 sampled at pixel centres (the edge width scales
    with R, so the images for R and 2R are the same shape at two scales), and its analytic
    gradient."""
    n = int(2 * R * (1 + margin * wf)) + 8
    c = (n - 1) / 2.0
    y, x = np.mgrid[0:n, 0:n].astype(np.float64)
    r = np.hypot(y - c, x - c)
    s = wf * R
    dudr = -0.5 / s / np.cosh((R - r) / s) ** 2
    rr = np.where(r > 0, r, 1.0)
    return 0.5 * (1 + np.tanh((R - r) / s)), dudr * (x - c) / rr, dudr * (y - c) / rr


def test_smooth_disk_sum_tends_to_the_axis_bias_term():
    """Sec. III-B states sampling and scale invariance of the continuum regulariser, but the
    discrete operator has only 8 normal directions (the axis bias Sec. V-B mentions): on an
    affine patch U = a x + b y its value is min(2|a|/3, 2|b|/3, |a+b|/2, |a-b|/2) (the affine
    closed form), not 0.  Along a disk's edge the gradient turns through every direction, so
    sum |H^w| grows with the perimeter, and for smooth disks it tends to the affine closed form
    applied to the analytic gradient, the remainder (the curvature terms) falling like 1/R.
    The scale-invariance claim itself is therefore not a property of the discrete method and is
    not pinned; this pins what the discrete method does instead."""
    ratios = []
    for R in (64, 128, 256):
        u, a, b = smooth_disk(R)
        g = np.minimum(np.minimum(2 * np.abs(a) / 3, 2 * np.abs(b) / 3),
                       np.minimum(np.abs(a + b) / 2, np.abs(a - b) / 2))
        ratios.append(oracle.energies(u)[0] / g.sum())
    assert 0.8 < ratios[0] < ratios[1] < ratios[2] < 1.0, ratios
    for k in range(2):
        shrink = (1 - ratios[k + 1]) / (1 - ratios[k])
        assert 0.35 < shrink < 0.7, (ratios, shrink)  # about 1/2 per doubling of R


# ------------------------------------------------------------ point-sampled forms of the oracle
def _points_with_borders(h, w, n, seed):
    """n random pixels plus every corner and a run along each of the four borders."""
    rng = np.random.default_rng(seed)
    ys = [rng.integers(0, h, n)]
    xs = [rng.integers(0, w, n)]
    for y, x in [(0, 0), (0, w - 1), (h - 1, 0), (h - 1, w - 1)]:
        ys.append(np.array([y]))
        xs.append(np.array([x]))
    k = min(w, 17)
    ys += [np.zeros(k, int), np.full(k, h - 1)]
    xs += [rng.integers(0, w, k), rng.integers(0, w, k)]
    k = min(h, 17)
    ys += [rng.integers(0, h, k), rng.integers(0, h, k)]
    xs += [np.zeros(k, int), np.full(k, w - 1)]
    return np.concatenate(ys), np.concatenate(xs)


@pytest.mark.parametrize("boundary", ["zero", "replicate"])
@pytest.mark.parametrize("shape", [(1, 1), (1, 9), (8, 1), (3, 4), (37, 53)])
def test_eval_points_match_the_appendix_on_integer_images(boundary, shape):
    """The point-sampled evaluation (the checker of every full-size GPU test) against the
    Appendix restatement through scipy's conv2, bit for bit on integer images (exact on both
    sides), at random pixels, all four corners and runs along all four borders."""
    rng = np.random.default_rng(sum(shape) + len(boundary))
    u = rng.integers(-40, 41, size=shape).astype(np.float64)
    want, dist = _appendix_wmc(u, boundary)
    ys, xs = _points_with_borders(*shape, 200, seed=sum(shape))
    got, cand = oracle.eval_points(u, ys, xs, boundary, candidates=True)
    assert np.array_equal(got, want[ys, xs])
    assert np.array_equal(np.sort(cand, -1), np.sort(dist[ys, xs], -1))


@pytest.mark.parametrize("boundary", ["zero", "replicate"])
def test_eval_points_equal_the_whole_image_oracle(boundary):
    """Real-valued image of non-square shape: the point-sampled values and candidates equal the
    whole-image oracle's at the same pixels, bit for bit (a transposed index or a wrong pitch in
    the sampled loop would move every value)."""
    u = synth.make_image(61, 47, seed=40, sigma=0.07).astype(np.float64)
    hw, cand, _ = oracle.wmc_eval(u, boundary, candidates=True)
    ys, xs = _points_with_borders(61, 47, 500, seed=41)
    got, c = oracle.eval_points(u, ys, xs, boundary, candidates=True)
    assert np.array_equal(got, hw[ys, xs])
    assert np.array_equal(c, cand[ys, xs])


@pytest.mark.parametrize("boundary", ["zero", "replicate"])
def test_step_points_equal_one_oracle_step(boundary):
    """One Jacobi step at sampled pixels (Sec. V-B, A = I; and Eq. MCF with mu = 0) equals one
    whole-image oracle step from the same U^t, bit for bit, at random pixels and on all borders."""
    f = synth.make_image(43, 58, seed=42, sigma=0.1).astype(np.float64)
    U = oracle.denoise(f, 1.3, 0.2, 3, boundary)
    ys, xs = _points_with_borders(43, 58, 400, seed=43)
    want = oracle.denoise(f, 1.3, 0.2, 1, boundary, u0=U)
    got = oracle.step_points(U, f, 1.3, 0.2, ys, xs, boundary)
    assert np.array_equal(got, want[ys, xs])
    want = oracle.mcf(U, 0.3, 1, boundary)
    got = oracle.step_points(U, None, 1.0, 0.3, ys, xs, boundary, mu=0.0)
    assert np.array_equal(got, want[ys, xs])


def test_step_points_by_hand():
    """The one-step example worked by hand above (a single 1 in a 3 x 3 image, lambda 1, step
    1/4): 0.75 at the centre, 0 elsewhere, here from the point-sampled step."""
    f = np.zeros((3, 3))
    f[1, 1] = 1
    ys, xs = np.divmod(np.arange(9), 3)
    got = oracle.step_points(f, f, 1.0, 0.25, ys, xs)
    want = np.zeros(9)
    want[4] = 0.75
    assert np.array_equal(got, want)


# ----------------------------------------------------------------- harmonic quadratics
def _tangent_candidates(a, b):
    """Candidates d_1..d_8 of the affine image U = a x + b y (x = column, y = row down), derived
    by hand from the printed half windows: d1 = -2a/3, d2 = -2b/3, d3 = 2a/3, d4 = 2b/3,
    d5 = -(a+b)/2, d6 = (a-b)/2, d7 = (a+b)/2, d8 = -(a-b)/2."""
    return np.stack([-2 * a / 3, -2 * b / 3, 2 * a / 3, 2 * b / 3, -(a + b) / 2, (a - b) / 2,
                     (a + b) / 2, -(a - b) / 2], -1)


@pytest.mark.parametrize("which", ["xy", "x2-y2"])
def test_harmonic_quadratics_reduce_to_their_tangent_plane(which):
    """U = x y and U = x^2 - y^2 (harmonic, so the isotropic Laplacian of Eq. kernel3 is 0).
    Worked by hand from the printed kernels: the second-order part (dx dy, resp. dx^2 - dy^2)
    sums to zero over every one of the eight half windows, so at each interior pixel the eight
    d_i are exactly those of the tangent plane, gradient (y, x) for x y and (2x, -2y) for
    x^2 - y^2.  Hence |H^w| = min(2|a|/3, 2|b|/3, |a+b|/2, |a-b|/2) of that gradient, which is 0
    exactly where the gradient lies along one of the 8 discrete normals (the axes and the
    diagonals through the origin), and not 0 elsewhere."""
    y, x = np.mgrid[-6:7, -7:8].astype(np.float64)
    if which == "xy":
        u, a, b = x * y, y, x
    else:
        u, a, b = x ** 2 - y ** 2, 2 * x, -2 * y
    for boundary in ("replicate", "zero"):
        hw, cand, _ = oracle.wmc_eval(u, boundary, candidates=True)
        inner = (slice(1, -1), slice(1, -1))
        want = _tangent_candidates(a, b)[inner]
        assert np.array_equal(cand[inner] * 12, want * 12)  # all integers or halves: exact
        mag = np.minimum.reduce([2 * np.abs(a) / 3, 2 * np.abs(b) / 3, np.abs(a + b) / 2,
                                 np.abs(a - b) / 2])[inner]
        np.testing.assert_allclose(np.abs(hw[inner]), mag, rtol=0, atol=1e-14)
        zero = ((a == 0) | (b == 0) | (np.abs(a) == np.abs(b)))[inner]
        assert np.all(hw[inner][zero] == 0) and np.all(hw[inner][~zero] != 0)


# ------------------------------------------------------------------ tie events of Eq. act
def test_tie_count_on_ramps_impulses_and_steps():
    """Worked by hand from the printed kernels.  On the ramp x + 2y every interior pixel's
    candidates are +-1/2, +-1, +-2/3, +-4/3 (the closed form above with a = 1, b = 2): the least
    magnitude 1/2 comes with both signs, an opposite-sign tie; the border rows and columns under
    REPLICATE are not (e.g. 1/4 alone at the top-left corner, or a zero).  An impulse has no
    tie anywhere (every candidate at the centre is -1, and around it the least magnitude is a
    single 0), nor has a straight step edge (least magnitude 0)."""
    y, x = np.mgrid[0:9, 0:11].astype(np.float64)
    ramp = x + 2 * y
    _, cand, _ = oracle.wmc_eval(ramp, "replicate", candidates=True)
    mags = np.abs(cand)
    in_set = mags <= mags.min(-1, keepdims=True)
    both = (in_set & (cand > 0)).any(-1) & (in_set & (cand < 0)).any(-1)
    assert both[1:-1, 1:-1].all()
    assert oracle.count_ties(ramp, 0.0) == int(both.sum()) >= 7 * 9
    imp = np.zeros((7, 7))
    imp[3, 3] = 1.0
    assert oracle.count_ties(imp, 0.0) == 0
    assert oracle.count_ties((x >= 5) * 1.0, 0.0) == 0
    # the band widens with tau: candidates 1/2 and -2/3 of the ramp are within 1/6
    assert oracle.count_ties(ramp, 0.2) >= oracle.count_ties(ramp, 0.0)
    assert oracle.count_ties(-ramp, 0.0) == oracle.count_ties(ramp, 0.0)
