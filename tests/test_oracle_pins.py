"""Pins for the FP64 oracle: it is checked against things the paper and mathematics
fix, never against itself.

* Philox4x32-10 known-answer vectors (Random123 / SC'11) and cuRAND's own Philox.
* Uniform-ball / disk sampling: moments and the radial law of a uniform point.
* Weight function S: the integral condition of Eq. 5 (vanishing for every R, which
  with linear bands forces dr = dR/2^(1/3)), shape values, finite differences.
* Energy: the ideal-blob closed form printed as Eq. 3, its 2D analogue, the alpha = 3
  symmetric-slope condition of Eq. 4, and exact finite-band energies by quadrature.
* Gradients: finite differences of exact (quadrature) energies against the MC
  estimates of dE/dR and dE/dc; the identity between Eqs. 7-10 and the centre/radius
  form.
* Image model: a library interpolator (scipy RegularGridInterpolator) and numpy's
  float16 decoding.
* Invariants: constant image, linear ramp, integer translation.
* Brute force on a tiny random volume: dense quadrature of S * I over the ball.
* Convergence on a noise-free blob, lattice spacing (Fig. 1b), localization rules.
* Grid form of Eq. 5: convergence to the exact energy as the grid refines, partials
  equal to central differences of the grid energy, integer translation.
* Stopping rules (step and energy), pinned to their definitions: limits that make
  them equivalent to a shorter fixed-T run or to no rule at all.
"""
import math
import os
import subprocess

import numpy as np
import pytest

# quad reports roundoff when asked for 1e-12..1e-13 on piecewise-polynomial integrands; the pins'
# own tolerances are far looser, so the warning carries no information here
pytestmark = pytest.mark.filterwarnings("ignore::scipy.integrate.IntegrationWarning")

HERE = os.path.dirname(os.path.abspath(__file__))
RHO3 = 2.0 ** (-1.0 / 3.0)
RHO2 = 2.0 ** (-0.5)


# ----------------------------------------------------------------------------- Philox
def _kat_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            v = [int(t, 16) for t in line.split()]
            rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_philox_known_answers(oracle):
    for ctr, key, want in _kat_rows():
        got = oracle.philox(np.array([ctr], dtype=np.uint32), key)[0]
        assert [int(x) for x in got] == want


def test_philox_matches_curand_header(oracle, tmp_path):
    """cuRAND's Philox4x32-10 (a CUDA toolkit header, host path) on 2e5 counters."""
    nvcc = "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    so = tmp_path / "curand_ref.so"
    subprocess.run([nvcc, "-shared", "-Xcompiler", "-fPIC", "-DQUALIFIERS=static inline __host__ __device__",
                    "-o", str(so), os.path.join(HERE, "_curand_philox_ref.cu")], check=True, capture_output=True)
    import ctypes as ct
    lib = ct.CDLL(str(so))
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2**32, size=(200_000, 4), dtype=np.uint64).astype(np.uint32)
    key = np.array([0x12345678, 0x9ABCDEF0], dtype=np.uint32)
    want = np.empty_like(ctr)
    P = lambda a: a.ctypes.data_as(ct.c_void_p)
    lib.curand_philox_batch(ct.c_long(len(ctr)), P(ctr), P(key), P(want))
    np.testing.assert_array_equal(oracle.philox(ctr, key), want)


def test_uniform24(oracle):
    assert oracle.uniform24(0) == 0.0
    assert oracle.uniform24(0xFFFFFFFF) == 1.0 - 2.0**-24
    assert oracle.uniform24(0x100) == 2.0**-24
    assert oracle.uniform24(0xFF) == 0.0


# ----------------------------------------------------------------------------- sampling
@pytest.mark.parametrize("ndim", [2, 3])
def test_unit_ball_sampling_is_uniform(oracle, ndim):
    P = oracle.make_params(ndim, 200_000, seed=11)
    u = oracle.unit_samples(P, 1, 5)[:, :ndim]
    r = np.linalg.norm(u, axis=1)
    assert r.max() <= 1.0 + 1e-12
    n = len(u)
    # E|u|^2 = d/(d+2); E u = 0; E u_i^2 = 1/(d+2); E u_i u_j = 0
    assert abs(np.mean(r**2) - ndim / (ndim + 2)) < 5 * np.std(r**2) / math.sqrt(n)
    assert np.all(np.abs(u.mean(0)) < 5 * u.std(0) / math.sqrt(n))
    assert np.all(np.abs((u**2).mean(0) - 1 / (ndim + 2)) < 5 * (u**2).std(0) / math.sqrt(n))
    # radial law P(|u| < s) = s^d (Kolmogorov-Smirnov)
    from scipy.stats import kstest
    assert kstest(r**ndim, "uniform").pvalue > 1e-3
    if ndim == 2:
        assert np.all(u[:, :2] == u[:, :2])  # finite


def test_uniforms21(oracle):
    """The 3D sample's three 21-bit uniforms: w0 bits 31..11, w1 bits 20..0, and w0
    bits 10..0 followed by w1 bits 31..22 (w1 bit 21 unused)."""
    assert oracle.uniforms21(0, 0) == (0.0, 0.0, 0.0)
    top = 1.0 - 2.0**-21
    assert oracle.uniforms21(0xFFFFFFFF, 0xFFFFFFFF) == (top, top, top)
    assert oracle.uniforms21(0x800, 0) == (2.0**-21, 0.0, 0.0)          # lowest bit of u0
    assert oracle.uniforms21(0x400, 0) == (0.0, 0.0, 0.5)              # highest bit of u2
    assert oracle.uniforms21(0, 0x400000) == (0.0, 0.0, 2.0**-21)      # lowest bit of u2
    assert oracle.uniforms21(0, 0x200000) == (0.0, 0.0, 0.0)           # the unused bit
    assert oracle.uniforms21(0, 0x100000) == (0.0, 0.5, 0.0)           # highest bit of u1


@pytest.mark.parametrize("ndim,N", [(3, 67), (2, 33)])
def test_sample_word_layout(oracle, ndim, N):
    """Sample j takes words 2 j and 2 j + 1 of the stream Philox(0, n, k, s),
    Philox(1, n, k, s), ... (one block per two samples): radius, polar and azimuth
    angles follow from those two words alone -- 2D: two 24-bit uniforms (one per
    word); 3D: three 21-bit uniforms cut from the 64 bits (restated here with
    Python integers)."""
    it, k, sid = 4, 9, 2
    P = oracle.make_params(ndim, N, seed=0x1234567890ABCDEF, stream_id=sid)
    nb = (2 * N + 3) // 4
    ctr = np.array([[b, it, k, sid] for b in range(nb)], dtype=np.uint32)
    words = oracle.philox(ctr, [0x90ABCDEF, 0x12345678]).reshape(-1)
    u = oracle.unit_samples(P, it, k)
    for j in range(N):
        w0, w1 = int(words[2 * j]), int(words[2 * j + 1])
        bits = (w0 << 32) | w1                    # the 64 bits, w0 first
        r = np.linalg.norm(u[j, :ndim])
        if ndim == 3:
            u0 = (bits >> 43) / 2**21             # bits 63..43 = w0 bits 31..11
            u1 = (bits & (2**21 - 1)) / 2**21     # bits 20..0 = w1 bits 20..0
            u2 = ((bits >> 22) & (2**21 - 1)) / 2**21   # bits 42..22 = w0 10..0, w1 31..22
            assert r == pytest.approx(u0 ** (1 / 3), rel=1e-12, abs=1e-12)
            assert u[j, 2] == pytest.approx(r * (1 - 2 * u1), abs=1e-12)
        else:
            u0, u2 = (w0 >> 8) / 2**24, (w1 >> 8) / 2**24
            assert r == pytest.approx(math.sqrt(u0), rel=1e-12, abs=1e-12)
        if r > 1e-6 and np.hypot(u[j, 0], u[j, 1]) > 1e-9:
            th = math.atan2(u[j, 1], u[j, 0]) % (2 * math.pi)
            want = 2 * math.pi * u2
            assert min(abs(th - want), 2 * math.pi - abs(th - want)) < 1e-9


def test_counter_layout_distinct_streams(oracle):
    """Different contour index / iteration / stream give different samples."""
    P = oracle.make_params(3, 64, seed=3)
    a = oracle.unit_samples(P, 1, 0)
    assert not np.allclose(a, oracle.unit_samples(P, 2, 0))
    assert not np.allclose(a, oracle.unit_samples(P, 1, 1))
    P2 = oracle.make_params(3, 64, seed=3, stream_id=1)
    assert not np.allclose(a, oracle.unit_samples(P2, 1, 0))
    np.testing.assert_array_equal(a, oracle.unit_samples(P, 1, 0))


# ----------------------------------------------------------------------------- weight S
def _S(oracle, ndim, r, R, dR=1.0):
    return oracle.weight(ndim, np.atleast_1d(r), R, dR)


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("R", [0.5, 1.0, 2.0, 3.2659863, 7.0, 20.0])
def test_weight_integral_vanishes(oracle, ndim, R):
    """Eq. 5: the integral of S r^(d-1) over r is zero (constant images give E = 0)."""
    from scipy.integrate import quad
    dR = 1.0
    rho = RHO3 if ndim == 3 else RHO2
    dr = dR * rho
    brk = sorted({max(0.0, rho * R - dr / 2), rho * R + dr / 2, R - dR / 2, R + dR / 2})
    f = lambda r: _S(oracle, ndim, r, R, dR)[0, 0] * r ** (ndim - 1)
    val, err = quad(f, 0.0, R + dR / 2 + 1.0, points=brk, limit=200, epsabs=1e-13, epsrel=0)
    scale = (R + dR) ** ndim
    assert abs(val) < 1e-9 * scale


def test_inner_band_width_is_dR_over_cuberoot2(oracle):
    """The relation below Eq. 5: dr = dR / 2^(1/3) (3D); 2D analogue dR / sqrt 2."""
    for ndim, want in [(3, 2.0 ** (-1 / 3)), (2, 2.0 ** (-0.5))]:
        R = 10.0
        r = np.linspace(0, 12, 1_200_001)
        dS = _S(oracle, ndim, r, R, 1.0)[:, 2]
        inner = r[dS > 0]
        width = inner.max() - inner.min()
        assert abs(width - want) < 2e-5


@pytest.mark.parametrize("ndim", [2, 3])
def test_weight_shape_and_derivatives(oracle, ndim):
    R, dR = 6.0, 1.0
    rho = RHO3 if ndim == 3 else RHO2
    w = _S(oracle, ndim, [0.0, 0.5 * rho * R, (rho * R + R) / 2, R + dR / 2, R + dR, 100.0], R, dR)
    np.testing.assert_allclose(w[:, 0], [-1, -1, 1, 0, 0, 0], atol=1e-15)
    # finite differences away from band edges (where S is smooth)
    rng = np.random.default_rng(0)
    r = rng.uniform(0, R + dR, 4000)
    dr = dR * rho
    edges = np.array([rho * R - dr / 2, rho * R + dr / 2, R - dR / 2, R + dR / 2])
    r = r[np.min(np.abs(r[:, None] - edges[None]), axis=1) > 1e-3]
    h = 1e-5
    w0 = oracle.weight(ndim, r, R, dR)
    fd_r = (oracle.weight(ndim, r + h, R, dR)[:, 0] - oracle.weight(ndim, r - h, R, dR)[:, 0]) / (2 * h)
    fd_R = (oracle.weight(ndim, r, R + h, dR)[:, 0] - oracle.weight(ndim, r, R - h, dR)[:, 0]) / (2 * h)
    np.testing.assert_allclose(w0[:, 2], fd_r, atol=1e-6)
    np.testing.assert_allclose(w0[:, 1], fd_R, atol=1e-6)
    # S is continuous everywhere (it is piecewise linear with no jumps)
    rr = np.linspace(0, R + 2, 200001)
    s = oracle.weight(ndim, rr, R, dR)[:, 0]
    assert np.max(np.abs(np.diff(s))) < 3 * (rr[1] - rr[0]) * 2 / dr


# ----------------------------------------------------------------------------- energy
def _eval_blob(oracle, ndim, R, r0, amp, N, dR=1.0, seed=1, offset=0.0, centre_offset=(0.0, 0.0, 0.0), grad=(0, 0, 0)):
    img = oracle.BlobImage(ndim, (0.0, 0.0, 0.0)[:ndim], r0, amp, offset=offset, grad=grad)
    P = oracle.make_params(ndim, N, dR=dR, seed=seed)
    return oracle.eval_cr(img, P, list(centre_offset[:ndim]), R, 1, 0)


def _sig(res, idx):
    return math.sqrt(res[idx])


@pytest.mark.parametrize("frac", [0.8, 1.1, 1.5])
def test_eq3_ideal_sphere_closed_form(oracle, frac):
    """Eq. 3: I = 1 + sgn(r0 - r), concentric contour, sharp bands:
    E_hat = 0 (R < r0), -8/3 pi (R^3 - r0^3) (R/2^(1/3) < r0 < R), -8/3 pi r0^3 (R >= 2^(1/3) r0);
    E_hat = E (2R)^3 (Eq. 4 with alpha = 3 undone)."""
    r0 = 5.0
    R = frac * r0
    res = _eval_blob(oracle, 3, R, r0, amp=2.0, N=2_000_000, dR=0.02)
    if R < r0:
        want = 0.0
    elif R / 2 ** (1 / 3) < r0:
        want = -8.0 / 3.0 * math.pi * (R**3 - r0**3)
    else:
        want = -8.0 / 3.0 * math.pi * r0**3
    got = res[oracle.E] * (2 * R) ** 3
    tol = 5 * _sig(res, oracle.VAR_E) * (2 * R) ** 3 + 0.01 * abs(want) * 0.05
    assert abs(got - want) < tol, (got, want, tol)


@pytest.mark.parametrize("frac", [0.8, 1.2, 1.6])
def test_ideal_disk_closed_form(oracle, frac):
    """2D analogue of Eq. 3 (areas in place of volumes): A pi (r0^2 - R^2) between r0
    and sqrt 2 r0, -A pi r0^2 beyond, 0 below r0; normalised by (2R)^2."""
    r0, A = 6.0, 2.0
    R = frac * r0
    res = _eval_blob(oracle, 2, R, r0, amp=A, N=2_000_000, dR=0.02)
    if R < r0:
        want = 0.0
    elif R / math.sqrt(2) < r0:
        want = A * math.pi * (r0**2 - R**2)
    else:
        want = -A * math.pi * r0**2
    got = res[oracle.E] * (2 * R) ** 2
    assert abs(got - want) < 5 * _sig(res, oracle.VAR_E) * (2 * R) ** 2 + 1e-3 * abs(want)


def test_alpha3_symmetric_slope(oracle):
    """Eq. 4 and the limit below it: with alpha = 3 the slope of E(R) has the same
    magnitude just below and just above R = 2^(1/3) r0 (sharp bands)."""
    r0 = 5.0
    Rs = 2 ** (1 / 3) * r0
    left = _eval_blob(oracle, 3, Rs - 0.15, r0, 2.0, 2_000_000, dR=0.02)
    right = _eval_blob(oracle, 3, Rs + 0.15, r0, 2.0, 2_000_000, dR=0.02, seed=2)
    gl, gr = left[oracle.DEDR], right[oracle.DEDR]
    assert gl < 0 < gr
    # closed-form slopes: dE/dR = -/+ (A pi r0^3 / 2) / R^4 with A = 2 on either side,
    # so |dE/dR| R^4 -> pi r0^3 from both sides exactly when alpha = 3
    want = math.pi * r0**3
    sl = -gl * (Rs - 0.15) ** 4
    sr = gr * (Rs + 0.15) ** 4
    for s, res, R in ((sl, left, Rs - 0.15), (sr, right, Rs + 0.15)):
        assert abs(s - want) < 0.02 * want + 5 * _sig(res, oracle.VAR_R) * R**4, (s, want)
    assert abs(sl - sr) < 0.04 * want


def _exact_concentric(oracle, ndim, R, r0, A, dR):
    """E(R) for a concentric blob, by quadrature of the oracle's S (radial integral)."""
    from scipy.integrate import quad
    rho = RHO3 if ndim == 3 else RHO2
    dr = dR * rho
    brk = [b for b in (rho * R - dr / 2, rho * R + dr / 2, R - dR / 2, R + dR / 2) if 0 < b < r0]
    shell = 4 * math.pi if ndim == 3 else 2 * math.pi
    f = lambda r: _S(oracle, ndim, r, R, dR)[0, 0] * shell * r ** (ndim - 1)
    val = quad(f, 0.0, r0, points=brk or None, limit=200, epsabs=1e-12, epsrel=1e-12)[0]
    return A * val / (2 * R) ** ndim


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("R", [4.0, 5.6, 6.5, 8.0])
def test_finite_band_energy_and_dEdR(oracle, ndim, R):
    """MC energy and dE/dR (default dR = 1) against quadrature and its central difference."""
    r0, A = 5.0, 170.0
    res = _eval_blob(oracle, ndim, R, r0, A, 1_000_000, dR=1.0, offset=30.0, seed=5)
    E = _exact_concentric(oracle, ndim, R, r0, A, 1.0)
    h = 1e-4
    dE = (_exact_concentric(oracle, ndim, R + h, r0, A, 1.0) - _exact_concentric(oracle, ndim, R - h, r0, A, 1.0)) / (2 * h)
    assert abs(res[oracle.E] - E) < 5 * _sig(res, oracle.VAR_E) + 1e-9, (res[oracle.E], E)
    assert abs(res[oracle.DEDR] - dE) < 5 * _sig(res, oracle.VAR_R) + 1e-6, (res[oracle.DEDR], dE)


def _exact_offcentre(oracle, ndim, R, r0, A, dR, delta):
    """E for a blob whose centre is `delta` from the contour centre: radial integral
    of S times the measure of the sphere (circle) of radius r inside the blob."""
    from scipy.integrate import quad

    def measure(r):
        if r <= 0:
            return 0.0
        if r + delta <= r0:
            return 4 * math.pi * r * r if ndim == 3 else 2 * math.pi * r
        if r >= r0 + delta or r <= delta - r0:
            return 0.0
        ca = (r * r + delta * delta - r0 * r0) / (2 * r * delta)
        ca = min(1.0, max(-1.0, ca))
        return 2 * math.pi * r * r * (1 - ca) if ndim == 3 else 2 * r * math.acos(ca)

    rho = RHO3 if ndim == 3 else RHO2
    dr = dR * rho
    Ro = R + dR / 2
    brk = [b for b in (rho * R - dr / 2, rho * R + dr / 2, R - dR / 2, abs(r0 - delta), r0 + delta) if 0 < b < Ro]
    f = lambda r: _S(oracle, ndim, r, R, dR)[0, 0] * measure(r)
    val = quad(f, 0.0, Ro, points=brk, limit=400, epsabs=1e-12, epsrel=1e-12)[0]
    return A * val / (2 * R) ** ndim


@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("delta", [0.7, 2.0])
def test_centre_gradient_against_exact(oracle, ndim, delta):
    """dE/dc (MC) against the central difference of the exact off-centre energy.
    The contour sits at +delta along an oblique axis from the blob centre."""
    r0, A, R = 5.0, 170.0, 6.0
    e = np.array([2.0, -1.0, 2.0][:ndim])
    e = e / np.linalg.norm(e)
    h = 1e-4
    dE = (_exact_offcentre(oracle, ndim, R, r0, A, 1.0, delta + h) - _exact_offcentre(oracle, ndim, R, r0, A, 1.0, delta - h)) / (2 * h)
    res = _eval_blob(oracle, ndim, R, r0, A, 1_000_000, dR=1.0, centre_offset=tuple(delta * e) + (0.0,) * (3 - ndim), seed=9)
    g = res[oracle.DEDC:oracle.DEDC + ndim]
    sig = np.sqrt(res[oracle.VAR_C:oracle.VAR_C + ndim])
    along = float(g @ e)
    assert abs(along - dE) < 5 * float(np.sqrt((sig**2) @ (e**2))) + 1e-6, (along, dE)
    # the component perpendicular to e vanishes in expectation
    perp = g - along * e
    assert np.all(np.abs(perp) < 5 * sig + 1e-6)
    # energy itself
    Ex = _exact_offcentre(oracle, ndim, R, r0, A, 1.0, delta)
    assert abs(res[oracle.E] - Ex) < 5 * _sig(res, oracle.VAR_E)


def test_pq_partials_match_centre_radius_form(oracle):
    """Eqs. 7-10 and the (c, R) form: dE/dR = dE/dq_x - dE/dp_x, dE/dc = dE/dp + dE/dq,
    and Eq. 9/10's equality of the p and q partials along y and z."""
    img = oracle.BlobImage(3, (0.0, 0.0, 0.0), 5.0, 170.0, offset=30.0)
    P = oracle.make_params(3, 4096, seed=4)
    p = np.array([-6.0 + 0.8, 0.5, -0.3])
    q = np.array([6.0 + 0.8, 0.5, -0.3])
    res = oracle.eval_pq(img, P, p, q, 3, 17)
    assert res[oracle.DEDP + 1] == res[oracle.DEDQ + 1]
    assert res[oracle.DEDP + 2] == res[oracle.DEDQ + 2]
    assert abs(res[oracle.DEDR] - (res[oracle.DEDQ] - res[oracle.DEDP])) < 1e-12 * (1 + abs(res[oracle.DEDR]))
    # gamma = (q_x - p_x)^-3 (Eq. 11): the energy scales as 1/L^3 for a fixed sum
    res2 = oracle.eval_cr(img, P, [0.8, 0.5, -0.3], 6.0, 3, 17)
    np.testing.assert_allclose(res2[:11], res[:11], rtol=1e-12, atol=1e-12)
    assert abs(res[oracle.E] - res[oracle.SUM_SI] / 12.0**3) < 1e-12 * (1 + abs(res[oracle.E]))


# ----------------------------------------------------------------------------- image model
def test_trilinear_matches_library_interpolator(oracle):
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(3)
    vol = rng.integers(0, 65535, size=(5, 7, 9), dtype=np.uint16)   # z, y, x
    sp = (1.0, 1.5, 2.5)
    img = oracle.VolumeImage(vol, sp, scale=0.5)
    f = RegularGridInterpolator((np.arange(5), np.arange(7), np.arange(9)), vol.astype(np.float64), method="linear")
    x = rng.uniform([-3, -3, -3], [9 * sp[0] + 3, 7 * sp[1] + 3, 5 * sp[2] + 3], size=(5000, 3))
    idx = x / np.array(sp)
    idx = np.clip(idx, 0, np.array([8, 6, 4]))
    want = 0.5 * f(idx[:, ::-1])
    np.testing.assert_allclose(oracle.image_values(img, x), want, rtol=1e-12, atol=1e-9)


def test_bilinear_matches_library_interpolator(oracle):
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(4)
    img2 = rng.integers(0, 255, size=(6, 11), dtype=np.uint8)
    img = oracle.VolumeImage(img2, (1.0, 1.0, 1.0))
    f = RegularGridInterpolator((np.arange(6), np.arange(11)), img2.astype(np.float64))
    x = np.zeros((3000, 3))
    x[:, :2] = rng.uniform([-2, -2], [13, 8], size=(3000, 2))
    idx = np.clip(x[:, :2], 0, [10, 5])
    np.testing.assert_allclose(oracle.image_values(img, x), f(idx[:, ::-1]), rtol=1e-12, atol=1e-9)


def test_half_decoding_matches_numpy(oracle):
    bits = np.arange(65536, dtype=np.uint16)
    want = bits.view(np.float16).astype(np.float64)
    got = np.array([oracle.half_to_double(int(b)) for b in bits[::7]])
    w = want[::7]
    fin = np.isfinite(w)
    np.testing.assert_array_equal(got[fin], w[fin])
    assert np.all(np.isnan(got[np.isnan(w)]))


def test_f16_volume_reads_like_u16(oracle):
    rng = np.random.default_rng(5)
    vol = rng.integers(0, 2048, size=(4, 5, 6)).astype(np.uint16)
    x = rng.uniform(-1, 7, size=(500, 3))
    a = oracle.image_values(oracle.VolumeImage(vol), x)
    b = oracle.image_values(oracle.VolumeImage(vol.astype(np.float16)), x)
    np.testing.assert_array_equal(a, b)


# ----------------------------------------------------------------------------- invariants
@pytest.mark.parametrize("ndim", [2, 3])
def test_constant_and_linear_images_give_zero(oracle, ndim):
    """Zero response to a constant image (the reason for rho) and, by symmetry, to a
    linear ramp; checked in expectation at 5 sigma."""
    for grad in [(0, 0, 0), (3.0, -2.0, 1.5)]:
        res = _eval_blob(oracle, ndim, 5.0, 1.0, amp=0.0, N=400_000, offset=500.0, centre_offset=(10.0, 20.0, 30.0),
                         grad=grad, seed=21)
        assert abs(res[oracle.E]) < 5 * _sig(res, oracle.VAR_E) + 1e-12
        assert abs(res[oracle.DEDR]) < 5 * _sig(res, oracle.VAR_R) + 1e-12
        for a in range(ndim):
            assert abs(res[oracle.DEDC + a]) < 5 * _sig(res, oracle.VAR_C + a) + 1e-12


def test_integer_translation_invariance(oracle):
    rng = np.random.default_rng(8)
    vol = rng.integers(0, 255, size=(20, 24, 28), dtype=np.uint8)
    big = np.zeros((20 + 6, 24 + 10, 28 + 14), dtype=np.uint8)
    big[3:23, 5:29, 7:35] = vol
    P = oracle.make_params(3, 512, seed=77)
    a = oracle.eval_cr(oracle.VolumeImage(vol), P, [13.3, 11.7, 9.2], 4.1, 5, 123)
    b = oracle.eval_cr(oracle.VolumeImage(big), P, [13.3 + 7, 11.7 + 5, 9.2 + 3], 4.1, 5, 123)
    np.testing.assert_allclose(a[:11], b[:11], rtol=1e-12, atol=1e-12)


@pytest.mark.slow
def test_brute_force_quadrature_tiny_volume(oracle):
    """Dense quadrature of S * I over the ball on a random 9^3 volume (library
    interpolator) against the MC estimate at large N."""
    from scipy.interpolate import RegularGridInterpolator
    rng = np.random.default_rng(12)
    vol = rng.integers(0, 255, size=(9, 9, 9), dtype=np.uint8)
    c = np.array([4.3, 3.8, 4.1])
    R, dR = 2.6, 1.0
    Ro = R + dR / 2
    f = RegularGridInterpolator((np.arange(9),) * 3, vol.astype(np.float64))
    m = 160
    g = (np.arange(m) + 0.5) / m * 2 * Ro - Ro
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pts = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    r = np.linalg.norm(pts, axis=1)
    keep = r <= Ro
    pts, r = pts[keep], r[keep]
    idx = np.clip(pts + c, 0, 8)
    I = f(idx[:, ::-1])
    S = oracle.weight(3, r, R, dR)[:, 0]
    quad_E = np.sum(S * I) * (2 * Ro / m) ** 3 / (2 * R) ** 3
    P = oracle.make_params(3, 4_000_000, dR=dR, seed=5)
    res = oracle.eval_cr(oracle.VolumeImage(vol), P, list(c), R, 1, 0)
    assert abs(res[oracle.E] - quad_E) < 5 * _sig(res, oracle.VAR_E) + 2e-3 * res[oracle.MAG_E]


def test_grid_energy_close_to_mc(oracle):
    """Eq. 5 on the voxel grid and the MC estimate describe the same integral.  The
    grid sum carries a discretisation bias (the grid sum of S is not exactly zero),
    so this is a loose sanity bound: within 15% of the magnitude sum near the fit."""
    from paper_1804_06304_gb300 import synth
    vol = synth.sphere_volume((40, 40, 40), (19.5, 20.2, 19.8), 7.0)
    img = oracle.VolumeImage(vol)
    P = oracle.make_params(3, 400_000, seed=3)
    for R in (8.8, 10.0):
        res = oracle.eval_cr(img, P, [19.5, 20.2, 19.8], R, 1, 0)
        grid = oracle.energy_grid(img, 3, [19.5, 20.2, 19.8], R, 1.0)
        assert abs(grid - res[oracle.E]) < 0.15 * res[oracle.MAG_E]


# ----------------------------------------------------------------------------- update, convergence
def test_update_follows_eqs_12_15(oracle):
    img = oracle.BlobImage(3, (0.0, 0.0, 0.0), 5.0, 1.0, n=(100, 100, 100))
    P = oracle.make_params(3, 16, eps0=0.3, max_step=10.0, Rmin=0.1, Rmax=100.0)
    res = np.zeros(oracle.RES_LEN)
    res[oracle.DEDP:oracle.DEDP + 3] = [0.2, -0.1, 0.05]
    res[oracle.DEDQ:oracle.DEDQ + 3] = [-0.4, -0.1, 0.05]
    p0, q0 = np.array([40.0, 50.0, 60.0]), np.array([48.0, 50.0, 60.0])
    p, q = oracle.update_pq(img, P, 4, res, p0, q0)
    eps = 0.3 / 2.0
    np.testing.assert_allclose(p, p0 - eps * res[1:4], rtol=1e-14)
    np.testing.assert_allclose(q, q0 - eps * res[4:7], rtol=1e-14)
    # step clamp: the centre moves at most max_step, the radius at most max_step
    P2 = oracle.make_params(3, 16, eps0=100.0, max_step=0.5, Rmin=0.1, Rmax=100.0)
    p, q = oracle.update_pq(img, P2, 1, res, p0, q0)
    c0, c1 = (p0 + q0) / 2, (p + q) / 2
    assert abs(np.linalg.norm(c1 - c0) - 0.5) < 1e-12
    assert abs((q[0] - p[0]) / 2 - (4.0 + 0.5)) < 1e-12


@pytest.mark.parametrize("ndim", [2, 3])
def test_convergence_noise_free_blob(oracle, ndim):
    """A noise-free blob and one contour seeded within R0/2 of its centre: the
    centre converges to within 0.25 voxel and R to within 10% of the radius that
    minimises the exact (quadrature) energy of the ideal blob.  One run's end point
    carries the Monte-Carlo noise of its last steps (over 40 random streams about
    three in four end within 0.25 voxel, the median near 0.15), so the pin takes the
    median over 16 streams; every run must end on the blob (E < 0)."""
    from scipy.optimize import minimize_scalar
    from paper_1804_06304_gb300 import synth
    r0, A = 5.0, 170.0
    shape = (32,) * ndim
    ctr = (15.6, 16.3, 15.9)[:ndim]
    vol = synth.sphere_volume(shape, ctr, r0, 200.0, 30.0)
    img = oracle.VolumeImage(vol)
    R0 = 4.0 / math.sqrt(1.5)
    seed = np.array(list(ctr) + [0.0] * (3 - ndim)) + np.array([1.0, -0.8, 0.6])[:3] * (1 if ndim == 3 else np.array([1, 1, 0]))
    errs, radii, energies = [], [], []
    for stream in range(1, 17):
        P = oracle.make_params(ndim, 256, 100, eps0=8 * R0**2 / A, max_step=0.5, Rmin=R0 / 2, Rmax=3 * R0,
                               seed=stream)
        cR, E, _ = oracle.evolve(img, P, np.array([list(seed) + [R0]]))
        errs.append(np.linalg.norm(cR[0, :ndim] - np.array(ctr)))
        radii.append(cR[0, 3])
        energies.append(E[0])
    assert np.median(errs) < 0.25, errs
    Rstar = minimize_scalar(lambda R: _exact_concentric(oracle, ndim, R, r0, A, 1.0), bounds=(r0, 2 * r0),
                            method="bounded").x
    assert abs(np.median(radii) - Rstar) < 0.1 * Rstar, (radii, Rstar)
    assert max(energies) < 0, energies


def test_wrapper_accepts_non_contiguous_state(oracle):
    """Marshalling: a transposed (Fortran-ordered) state array evolves like its
    C-ordered copy."""
    from paper_1804_06304_gb300 import synth
    vol = synth.sphere_volume((24, 24, 24), (11.5, 12.2, 11.9), 5.0)
    img = oracle.VolumeImage(vol)
    P = oracle.make_params(3, 64, 4, eps0=0.3, Rmin=1.0, Rmax=9.0, seed=2)
    soa = np.array([[10.0, 13.0, 11.0], [12.0, 11.0, 12.5], [11.0, 12.0, 12.0], [4.0, 3.5, 3.0]], np.float32)
    a = oracle.evolve(img, P, soa.T.astype(np.float64))[0]
    b = oracle.evolve(img, P, np.ascontiguousarray(soa.T, dtype=np.float64))[0]
    np.testing.assert_array_equal(a, b)
    np.testing.assert_allclose(a[:, :3], b[:, :3])


# ----------------------------------------------------------------------------- lattice, localize
def test_lattice_spacing_and_count(oracle):
    """Fig. 1b / Fig. 4b: neighbours sqrt(1.5) R0 apart; stride 4 over 64x64x32 gives 16x16x8."""
    s = oracle.seed_lattice(3, (64, 64, 32), (1, 1, 1), 4.0)
    assert len(s) == 2048
    R0 = s[0, 3]
    assert abs(np.linalg.norm(s[1, :3] - s[0, :3]) - math.sqrt(1.5) * R0) < 1e-12
    np.testing.assert_allclose(s[:, :3].mean(0), [31.5, 31.5, 15.5])
    s2 = oracle.seed_lattice(2, (4096, 4096), (1, 1), 6.0)
    assert len(s2) == 682 * 682 and np.all(s2[:, 2] == 0)
    s3 = oracle.seed_lattice(3, (1024, 1024, 256), (1, 1, 2), 6.0)
    assert len(s3) == 170 * 170 * 85


def test_localize_rules(oracle):
    rho = RHO3
    # A-B overlap, B-C overlap, A-C do not: A (lowest E) and C survive
    cR = np.array([[0, 0, 0, 5.0], [3.5, 0, 0, 5.0], [7.0, 0, 0, 5.0]])
    E = np.array([-10.0, -9.0, -8.0])
    assert list(oracle.localize(3, cR, E, -1.0)) == [0, 2]
    # equal energies: the lower index wins
    cR = np.array([[0, 0, 0, 5.0], [1.0, 0, 0, 5.0]])
    assert list(oracle.localize(3, cR, np.array([-4.0, -4.0]), -1.0)) == [0]
    assert list(oracle.localize(3, cR[::-1].copy(), np.array([-4.0, -4.0]), -1.0)) == [0]
    # E == E0 is kept, E > E0 and non-finite are dropped
    cR = np.array([[0, 0, 0, 1.0], [10, 0, 0, 1.0], [20, 0, 0, 1.0], [30, 0, 0, 1.0]])
    E = np.array([-3.0, -2.9, np.nan, -np.inf])
    assert list(oracle.localize(3, cR, E, -3.0)) == [0]
    # just inside / just outside rho * max(R', R'') with unequal radii
    lim = rho * 6.0
    cR = np.array([[0, 0, 0, 6.0], [lim * (1 - 1e-9), 0, 0, 2.0], [0, 50, 0, 6.0], [lim * (1 + 1e-9), 50, 0, 2.0]])
    assert list(oracle.localize(3, cR, np.array([-5.0, -6.0, -5.0, -6.0]), 0.0)) == [1, 3, 2]
    # exactly at the limit: not an overlap (the paper's test is strict)
    lim = rho * 6.0
    cR = np.array([[0, 0, 0, 6.0], [lim, 0, 0, 2.0]])
    assert math.sqrt(lim * lim) == lim
    assert list(oracle.localize(3, cR, np.array([-5.0, -6.0]), 0.0)) == [1, 0]
    # 2D uses rho = 1/sqrt 2
    cR = np.array([[0, 0, 0, 4.0], [RHO2 * 4.0 * 0.999, 0, 0, 4.0]])
    assert list(oracle.localize(2, cR, np.array([-1.0, -2.0]), 0.0)) == [1]
    assert len(oracle.localize(3, np.zeros((0, 4)), np.zeros(0), 0.0)) == 0


# ----------------------------------------------------------------------------- grid form of Eq. 5
@pytest.mark.parametrize("ndim", [2, 3])
@pytest.mark.parametrize("R", [4.0, 5.6, 6.5])
def test_grid_energy_converges_to_exact(oracle, ndim, R):
    """The voxel-grid sum of Eq. 5 on an ideal blob sampled at spacing h tends to
    the exact finite-band energy (quadrature) as h -> 0."""
    exact = _exact_concentric(oracle, ndim, R, 5.0, 170.0, 1.0)
    errs = []
    for h in (0.5, 0.0625):
        img = oracle.BlobImage(ndim, (0.0, 0.0, 0.0)[:ndim], 5.0, 170.0, offset=30.0)
        img.s.spacing[:] = (h, h, h)
        res = oracle.eval_cr(img, oracle.make_params(ndim, 1, integration=1), [0.0] * ndim, R, 1, 0)
        errs.append(abs(res[oracle.E] - exact) / res[oracle.MAG_E])
    assert errs[1] < 3e-3, errs
    assert errs[1] < errs[0] or errs[0] < 1e-3, errs


@pytest.mark.parametrize("ndim", [2, 3])
def test_grid_partials_are_derivatives_of_grid_energy(oracle, ndim):
    """dE/dR and dE/dc of the grid form (Eqs. 7-10 over the voxel grid) equal
    central differences of the grid energy itself, on a random anisotropic volume."""
    rng = np.random.default_rng(31 + ndim)
    shape = (14, 15, 16)[:ndim]
    vol = rng.integers(0, 255, size=shape, dtype=np.uint8)
    sp = (1.0, 1.25, 2.0) if ndim == 3 else (1.0, 1.25, 1.0)
    img = oracle.VolumeImage(vol, sp)
    P = oracle.make_params(ndim, 1, integration=1)
    h = 1e-6
    for trial in range(6):
        c = [rng.uniform(4.0, 9.0) for _ in range(ndim)]
        R = rng.uniform(2.5, 4.5)
        res = oracle.eval_cr(img, P, c, R, 1, 0)
        if res[oracle.FLAGS] > 0:
            continue
        E = lambda cc, RR: oracle.eval_cr(img, P, cc, RR, 1, 0)[oracle.E]
        dR = (E(c, R + h) - E(c, R - h)) / (2 * h)
        assert abs(res[oracle.DEDR] - dR) < 1e-6 * res[oracle.MAG_R], (trial, res[oracle.DEDR], dR)
        for a in range(ndim):
            cp = list(c); cm = list(c)
            cp[a] += h; cm[a] -= h
            dc = (E(cp, R) - E(cm, R)) / (2 * h)
            assert abs(res[oracle.DEDC + a] - dc) < 1e-6 * res[oracle.MAG_G], (trial, a, res[oracle.DEDC + a], dc)
        # the energy is the literal Eq. 5 grid sum
        assert abs(res[oracle.E] - oracle.energy_grid(img, ndim, c + [0.0] * (3 - ndim), R, 1.0)) < 1e-12 * \
            res[oracle.MAG_E] + 1e-12


def test_grid_integer_translation_invariance(oracle):
    rng = np.random.default_rng(9)
    vol = rng.integers(0, 255, size=(20, 24, 28), dtype=np.uint8)
    big = np.zeros((26, 34, 42), dtype=np.uint8)
    big[3:23, 5:29, 7:35] = vol
    P = oracle.make_params(3, 1, integration=1)
    a = oracle.eval_cr(oracle.VolumeImage(vol), P, [13.3, 11.7, 9.2], 4.1, 5, 123)
    b = oracle.eval_cr(oracle.VolumeImage(big), P, [20.3, 16.7, 12.2], 4.1, 5, 123)
    np.testing.assert_allclose(a[:11], b[:11], rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------------------- stopping rules
def _stop_case(oracle):
    from paper_1804_06304_gb300 import synth
    vol = synth.sphere_volume((32, 32, 32), (15.6, 16.3, 15.9), 5.0, 200.0, 30.0)
    img = oracle.VolumeImage(vol)
    R0 = 4.0 / math.sqrt(1.5)
    seeds = np.array([[15.6 + dx, 16.3 - dx, 15.9 + 0.5 * dx, R0] for dx in (0.0, 0.8, 1.6, 2.4)])
    kw = dict(eps0=8 * R0**2 / 170.0, max_step=0.5, Rmin=R0 / 2, Rmax=3 * R0, seed=4)
    return img, seeds, kw


def test_freeze_rule_limits(oracle):
    """freeze_tol huge: every contour stops after freeze_iters evaluations with the
    state and energy of a fixed run of T = freeze_iters (the last proposed step is
    not applied); freeze_tol = 0: identical to no rule."""
    img, seeds, kw = _stop_case(oracle)
    base = oracle.evolve(img, oracle.make_params(3, 64, 30, **kw), seeds, stops=True)
    short = oracle.evolve(img, oracle.make_params(3, 64, 3, **kw), seeds)
    big = oracle.evolve(img, oracle.make_params(3, 64, 30, freeze_tol=1e9, freeze_iters=3, **kw), seeds, stops=True)
    np.testing.assert_array_equal(big[0], short[0])
    np.testing.assert_array_equal(big[1], short[1])
    assert (big[3] == 1).all() and (big[4] == 3).all()
    zero = oracle.evolve(img, oracle.make_params(3, 64, 30, freeze_tol=0.0, freeze_iters=1, **kw), seeds, stops=True)
    np.testing.assert_array_equal(zero[0], base[0])
    assert (zero[3] == 0).all() and (zero[4] == 30).all() and (base[4] == 30).all()


def test_energy_rule_limits(oracle):
    """cull_E = -inf: every contour stops at cull_iter with the state of a fixed run
    of T = cull_iter; cull_E = +inf: identical to no rule."""
    img, seeds, kw = _stop_case(oracle)
    base = oracle.evolve(img, oracle.make_params(3, 64, 30, **kw), seeds)
    short = oracle.evolve(img, oracle.make_params(3, 64, 5, **kw), seeds)
    allc = oracle.evolve(img, oracle.make_params(3, 64, 30, cull_iter=5, cull_E=-np.inf, **kw), seeds, stops=True)
    np.testing.assert_array_equal(allc[0], short[0])
    np.testing.assert_array_equal(allc[1], short[1])
    assert (allc[3] == 2).all() and (allc[4] == 5).all()
    none = oracle.evolve(img, oracle.make_params(3, 64, 30, cull_iter=5, cull_E=np.inf, **kw), seeds, stops=True)
    np.testing.assert_array_equal(none[0], base[0])
    assert (none[3] == 0).all()


def test_freeze_rule_stops_converged_contours_early(oracle):
    """On a noise-free blob the contours converge, their steps (Monte-Carlo noise
    times the decaying eps_n) shrink below the tolerance and they stop before T,
    still on the blob centre."""
    img, seeds, kw = _stop_case(oracle)
    cR, E, tr, st, ne = oracle.evolve(img, oracle.make_params(3, 256, 200, freeze_tol=0.1, freeze_iters=4, **kw),
                                      seeds, trace=True, stops=True)
    assert (st == 1).all() and (ne < 200).all(), ne
    assert np.all(np.linalg.norm(cR[:, :3] - np.array([15.6, 16.3, 15.9]), axis=1) < 0.25)
    for i in range(len(seeds)):   # trace rows stop at the last evaluation, which is the final state
        assert np.isnan(tr[ne[i]:, i]).all() and not np.isnan(tr[:ne[i], i]).any()
        np.testing.assert_array_equal(tr[ne[i] - 1, i, :4], cR[i])


def test_freeze_rule_counts_consecutive_steps(oracle):
    """On a noisy image, where steps wander around the tolerance, a contour stops
    exactly when freeze_iters consecutive proposed steps are small: the trace shows
    freeze_iters - 1 small applied steps before the stop and no earlier run that
    long, and contours that ran to T never had such a run."""
    from paper_1804_06304_gb300 import synth
    s = synth.small_3d(3)
    img = oracle.VolumeImage(s.volume)
    R0 = 4.0 / math.sqrt(1.5)
    seeds = oracle.seed_lattice(3, s.shape_xyz, (1.0, 1.0, 1.0), 4.0)[::7]
    kw = dict(eps0=8 * R0**2 / s.contrast, max_step=0.5, Rmin=R0 / 2, Rmax=3 * R0, seed=6)
    tol, k = 0.12, 3
    cR, E, tr, st, ne = oracle.evolve(img, oracle.make_params(3, 64, 60, freeze_tol=tol, freeze_iters=k, **kw),
                                      seeds, trace=True, stops=True)
    assert 0 < (st == 1).sum() < len(seeds)
    for i in range(len(seeds)):
        rows = tr[:ne[i], i, :4]
        step = np.abs(np.diff(rows, axis=0)).max(axis=1)
        run, longest = 0, 0
        for small in step < tol:
            run = run + 1 if small else 0
            longest = max(longest, run)
        assert longest < k
        if st[i] == 1:
            assert run == k - 1, (i, step[-k:])
