"""Seeded synthetic inputs for GMMNLSE propagation problems.

This module builds the *inputs* of the solver -- per-mode propagation
constants beta_p(omega), the mode-overlap coupling tensor S_plmn, the Raman
response h_R and the launched pulse A_p(0, t) -- for the fiber and pulse
configurations used by the tests and the benchmark.  It contains none of the
propagation arithmetic (no dispersion operator, no nonlinear term, no MPA
iteration): both the CUDA path and the CPU oracle receive the arrays made here.

Physics sources for the generators:
  * Eq. 1 (Sec. III): the dispersion operator is a Taylor series of beta_p(omega)
    about omega_0, written relative to the first mode (delta beta_0, delta
    beta_1 of mode 1 removed).
  * Eq. 2 (Sec. III): S_plmn = int F_p F_l F_m F_n / sqrt(prod int F^2), real
    scalar mode profiles in one linear polarisation.
  * Sec. III.A.1 / Sec. III.B.1: parabolic GRIN fibers have equally spaced mode
    groups (delta beta_0 = n P); their modes are Hermite-Gauss functions.
  * Sec. III.B.2: step-index fibers and their LP modes.
  * Sec. III.C.5: Raman response h_R, fraction f_R ~ 0.18 (values below).

Random numbers: SplitMix64 (Steele, Lea, Flood 2014) -> 53-bit uniforms ->
Box-Muller normals.  Everything is FP64 and deterministic for a given seed.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

C_LIGHT = 299792458.0  # m/s

# ----------------------------------------------------------------------------
# Random numbers
# ----------------------------------------------------------------------------
_MASK64 = (1 << 64) - 1


class SplitMix64:
    """SplitMix64 generator (Steele, Lea & Flood, OOPSLA 2014), pure integers."""

    def __init__(self, seed: int):
        self.state = seed & _MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & _MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Uniform in [0, 1) with 53 random bits."""
        return (self.next_u64() >> 11) * (1.0 / (1 << 53))

    def normals(self, count: int) -> np.ndarray:
        """Standard normals by the Box-Muller transform, generated in pairs."""
        out = []
        while len(out) < count:
            u1 = 1.0 - self.uniform()  # (0, 1]
            u2 = self.uniform()
            r = math.sqrt(-2.0 * math.log(u1))
            out.append(r * math.cos(2.0 * math.pi * u2))
            out.append(r * math.sin(2.0 * math.pi * u2))
        return np.array(out[:count], dtype=np.float64)


def random_mode_weights(num_modes: int, seed: int) -> np.ndarray:
    """Complex weights w_p = g_{2p} + i g_{2p+1}, normalised to sum |w_p|^2 = 1."""
    g = SplitMix64(seed).normals(2 * num_modes)
    w = g[0::2] + 1j * g[1::2]
    return w / math.sqrt(float(np.sum(np.abs(w) ** 2)))


def coupling_matrix(num_modes: int, scale: float, seed: int, symmetric: bool = True) -> np.ndarray:
    """Real linear mode coupling Q[n][p] [1/m] with normal entries times
    scale (symmetrised when `symmetric`, as a real index perturbation makes
    it), standing in for disorder coupling coefficients."""
    g = SplitMix64(seed).normals(num_modes * num_modes).reshape(num_modes, num_modes) * scale
    return 0.5 * (g + g.T) if symmetric else g


# ----------------------------------------------------------------------------
# Material and grids
# ----------------------------------------------------------------------------
def silica_index(lam_m):
    """Fused-silica refractive index from the three-term Sellmeier fit of
    Malitson (JOSA 55, 1205, 1965); wavelength in metres."""
    lam_um2 = (np.asarray(lam_m, dtype=np.float64) * 1e6) ** 2
    b = (0.6961663, 0.4079426, 0.8974794)
    c = (0.0684043 ** 2, 0.1162414 ** 2, 9.896161 ** 2)
    n2 = 1.0 + sum(bi * lam_um2 / (lam_um2 - ci) for bi, ci in zip(b, c))
    return np.sqrt(n2)


def omega_grid(nt: int, dt: float) -> np.ndarray:
    """Angular-frequency offsets from omega_0 in FFT order: 2 pi q / T for
    q < Nt/2, else 2 pi (q - Nt) / T, with T = Nt dt."""
    return 2.0 * np.pi * np.fft.fftfreq(nt, d=dt)


def time_grid(nt: int, dt: float) -> np.ndarray:
    """Sample times t_k = (k - Nt/2) dt of the launched field."""
    return (np.arange(nt, dtype=np.float64) - nt // 2) * dt


# ----------------------------------------------------------------------------
# Parabolic GRIN fiber: Hermite-Gauss modes, closed-form beta
# ----------------------------------------------------------------------------
def grin_mode_indices(num_modes: int):
    """HG_(mx,ny) indices ordered by group g = mx + ny ascending, then ny
    ascending within a group: HG00, HG10, HG01, HG20, HG11, HG02, ..."""
    out = []
    g = 0
    while len(out) < num_modes:
        for ny in range(g + 1):
            out.append((g - ny, ny))
        g += 1
    return out[:num_modes]


def grin_mode_width(radius: float, na: float, lam0: float) -> float:
    """1/e field radius of the fundamental mode of an infinite parabolic
    profile n^2(r) = n1^2 - NA^2 r^2 / a^2: w = sqrt(2 a / (k0 NA))."""
    k0 = 2.0 * np.pi / lam0
    return math.sqrt(2.0 * radius / (k0 * na))


def grin_beta_closed_form(omega_abs, group: int, radius: float, na: float):
    """beta_g(omega) = sqrt((omega n(omega)/c)^2 - 2 (g+1) (omega/c) NA / a),
    the harmonic-oscillator eigenvalue of the parabolic profile with NA held
    constant and the core index from the silica Sellmeier fit."""
    omega_abs = np.asarray(omega_abs, dtype=np.float64)
    lam = 2.0 * np.pi * C_LIGHT / omega_abs
    k = omega_abs * silica_index(lam) / C_LIGHT
    return np.sqrt(k * k - 2.0 * (group + 1) * (omega_abs / C_LIGHT) * na / radius)


def taylor_coefficients(beta_fn, omega0: float, order: int = 3, rel_step: float = 2e-3):
    """beta^(n)(omega0), n = 0..order, by FP64 central finite differences
    (fourth-order stencils, step rel_step*omega0)."""
    h = rel_step * omega0
    f = {k: float(beta_fn(omega0 + k * h)) for k in range(-3, 4)}
    d0 = f[0]
    d1 = (f[-2] - 8 * f[-1] + 8 * f[1] - f[2]) / (12 * h)
    d2 = (-f[-2] + 16 * f[-1] - 30 * f[0] + 16 * f[1] - f[2]) / (12 * h * h)
    d3 = (f[-3] - 8 * f[-2] + 13 * f[-1] - 13 * f[1] + 8 * f[2] - f[3]) / (8 * h ** 3)
    return [d0, d1, d2, d3][: order + 1]


def beta_from_taylor(coeffs_abs, omega):
    """Per-mode beta_p(omega) in the frame of mode 1 (Eq. 1): delta beta_0 and
    delta beta_1 are taken relative to mode 1, beta_n (n >= 2) kept as is.
    coeffs_abs: [N][order+1] absolute Taylor coefficients.  Returns [N][Nt]."""
    c = np.array(coeffs_abs, dtype=np.float64)
    rel = c.copy()
    rel[:, 0] -= c[0, 0]
    rel[:, 1] -= c[0, 1]
    out = np.zeros((c.shape[0], omega.size))
    for n in range(c.shape[1]):
        out += rel[:, n : n + 1] * omega[None, :] ** n / math.factorial(n)
    return out


def _hermite(n: int, x):
    return np.polynomial.hermite.hermval(x, [0] * n + [1])


def hg_profile_1d(n: int, x, w: float):
    """h_n(x) = H_n(sqrt(2) x / w) exp(-x^2/w^2) (unnormalised)."""
    return _hermite(n, math.sqrt(2.0) * x / w) * np.exp(-(x * x) / (w * w))


def hg_overlap_1d_gauss_hermite(nmax: int, w: float) -> np.ndarray:
    """X[a,b,c,d] = int h_a h_b h_c h_d dx / sqrt(prod int h_i^2 dx) for the
    1-D Hermite-Gauss factors, by Gauss-Hermite quadrature (exact: the
    integrands are polynomials times exp(-u^2))."""
    u, wq = np.polynomial.hermite.hermgauss(64)
    # int h_a h_b h_c h_d dx with u = 2x/w: dx = (w/2) du, sqrt(2) x / w = u/sqrt(2)
    H4 = np.array([_hermite(n, u / math.sqrt(2.0)) for n in range(nmax + 1)])
    quad4 = np.einsum("aq,bq,cq,dq,q->abcd", H4, H4, H4, H4, wq) * (w / 2.0)
    # int h_a^2 dx with v = sqrt(2) x / w: dx = (w/sqrt 2) dv
    H2 = np.array([_hermite(n, u) for n in range(nmax + 1)])
    norm2 = np.einsum("aq,aq,q->a", H2, H2, wq) * (w / math.sqrt(2.0))
    s = np.sqrt(norm2)
    return quad4 / (s[:, None, None, None] * s[None, :, None, None]
                    * s[None, None, :, None] * s[None, None, None, :])


def grin_S_gauss_hermite(modes, w: float) -> np.ndarray:
    """Eq. 2 for HG modes, separable: S = X(x-indices) * X(y-indices)."""
    nmax = max(max(m) for m in modes)
    X = hg_overlap_1d_gauss_hermite(nmax, w)
    mx = np.array([m[0] for m in modes])
    ny = np.array([m[1] for m in modes])
    Sx = X[np.ix_(mx, mx, mx, mx)]
    Sy = X[np.ix_(ny, ny, ny, ny)]
    return Sx * Sy


def overlap_tensor_from_profiles(F: np.ndarray, dA: float) -> np.ndarray:
    """Eq. 2 on a grid: F is [N][G] real profiles sampled on G points of area
    dA.  S_plmn = sum_g F_p F_l F_m F_n dA / sqrt(prod_i sum_g F_i^2 dA).
    Evaluated as a matrix product of the pair products F_p F_l over the grid."""
    N = F.shape[0]
    norms = np.sqrt(np.sum(F * F, axis=1) * dA)
    Fn = F / norms[:, None]
    pair = (Fn[:, None, :] * Fn[None, :, :]).reshape(N * N, -1)
    S = (pair @ pair.T) * dA
    return S.reshape(N, N, N, N)


def grin_S_grid(modes, w: float, radius: float, npts: int = 128, extent: float = 2.0):
    """Eq. 2 on an npts x npts grid over [-extent*a, extent*a]^2."""
    x = (np.arange(npts) - npts / 2 + 0.5) * (2 * extent * radius / npts)
    dx = x[1] - x[0]
    X, Y = np.meshgrid(x, x, indexing="ij")
    F = np.array([(hg_profile_1d(m, X, w) * hg_profile_1d(n, Y, w)).ravel() for m, n in modes])
    return overlap_tensor_from_profiles(F, dx * dx)


# ----------------------------------------------------------------------------
# Step-index fiber: weakly guiding LP modes
# ----------------------------------------------------------------------------
def _lp_eigen_u(ell: int, V: float):
    """Roots u in (0, V) of the weakly guiding LP characteristic equation
    u J_{l-1}(u) / J_l(u) + w K_{l-1}(w) / K_l(w) = 0, w = sqrt(V^2 - u^2),
    written as a continuous function via J_l(u) K_l(w) cross-multiplication:
    g(u) = u J_{l-1}(u) K_l(w) + w K_{l-1}(w) J_l(u)."""
    from scipy.optimize import brentq
    from scipy.special import jv, kv

    def g(u):
        wv = math.sqrt(max(V * V - u * u, 1e-300))
        return u * jv(ell - 1, u) * kv(ell, wv) + wv * kv(ell - 1, wv) * jv(ell, u)

    us = np.linspace(1e-6, V * (1 - 1e-9), 20000)
    ws = np.sqrt(np.maximum(V * V - us * us, 1e-300))
    vals = us * jv(ell - 1, us) * kv(ell, ws) + ws * kv(ell - 1, ws) * jv(ell, us)
    roots = []
    for i in np.nonzero(vals[:-1] * vals[1:] < 0)[0]:
        # g is continuous on (0, V), so every sign change brackets a root
        roots.append(brentq(g, us[i], us[i + 1], xtol=1e-15, rtol=1e-15, maxiter=200))
    return roots


def step_index_modes(radius: float, na: float, lam0: float, num_modes: int):
    """First num_modes LP modes (both cos and sin orientations for l >= 1),
    ordered by beta descending, cos before sin.  Returns a list of dicts with
    l, m, orientation, u, w and beta at lam0."""
    k0 = 2 * np.pi / lam0
    V = k0 * radius * na
    n_cl = float(silica_index(lam0))
    n_co = math.sqrt(n_cl ** 2 + na ** 2)
    found = []
    for ell in range(0, 200):
        us = _lp_eigen_u(ell, V)
        if not us:
            break
        for mi, u in enumerate(us):
            beta = math.sqrt((k0 * n_co) ** 2 - (u / radius) ** 2)
            orients = ("cos",) if ell == 0 else ("cos", "sin")
            for o in orients:
                found.append(dict(l=ell, m=mi + 1, orient=o, u=u,
                                  w=math.sqrt(V * V - u * u), beta=beta))
    found.sort(key=lambda d: (-d["beta"], d["orient"] != "cos"))
    return found[:num_modes], dict(V=V, n_co=n_co, n_cl=n_cl)


def step_index_profile(mode, radius: float, X, Y):
    from scipy.special import jv, kv
    r = np.hypot(X, Y)
    phi = np.arctan2(Y, X)
    ell, u, wv = mode["l"], mode["u"], mode["w"]
    inside = jv(ell, u * r / radius)
    with np.errstate(over="ignore", invalid="ignore"):
        outside = jv(ell, u) / kv(ell, wv) * kv(ell, wv * np.maximum(r, 1e-30) / radius)
    radial = np.where(r <= radius, inside, outside)
    ang = np.cos(ell * phi) if mode["orient"] == "cos" else np.sin(ell * phi)
    return radial * ang


def step_index_beta_coeffs(radius, na, lam0, modes, order=3, rel_step=2e-3):
    """Taylor coefficients of each LP mode's beta(omega): the characteristic
    equation is re-solved at 7 frequencies around omega0 (silica cladding,
    NA held constant) and differentiated by the same stencils as the GRIN
    closed form.  Roots are found once per (azimuthal order, frequency)."""
    omega0 = 2 * np.pi * C_LIGHT / lam0
    cache = {}

    def roots(ell, om):
        key = (ell, om)
        if key not in cache:
            V = om / C_LIGHT * radius * na
            cache[key] = _lp_eigen_u(ell, V)
        return cache[key]

    coeffs = []
    for md in modes:
        def beta_fn(om, md=md):
            lam = 2 * np.pi * C_LIGHT / om
            k = om / C_LIGHT
            n_cl = float(silica_index(lam))
            n_co = math.sqrt(n_cl ** 2 + na ** 2)
            u = roots(md["l"], float(om))[md["m"] - 1]
            return math.sqrt((k * n_co) ** 2 - (u / radius) ** 2)
        coeffs.append(taylor_coefficients(beta_fn, omega0, order, rel_step))
    return coeffs


# ----------------------------------------------------------------------------
# Raman response and pulses
# ----------------------------------------------------------------------------
def raman_response(nt: int, dt: float, tau1: float = 12.2e-15, tau2: float = 32e-15):
    """Single damped-oscillator Raman response sampled at t_k = k dt (causal,
    circular over the window), renormalised so that dt * sum_k h_k = 1:
    h(t) = ((tau1^2 + tau2^2) / (tau1 tau2^2)) exp(-t/tau2) sin(t/tau1)."""
    t = np.arange(nt, dtype=np.float64) * dt
    h = ((tau1 ** 2 + tau2 ** 2) / (tau1 * tau2 ** 2)) * np.exp(-t / tau2) * np.sin(t / tau1)
    return h / (dt * np.sum(h))


def pulse_shape(kind: str, t, fwhm: float):
    """Field envelope normalised to peak 1.  Intensity FWHM convention:
    sech: sech(t/T0), FWHM = 2 acosh(sqrt 2) T0; gaussian: exp(-t^2/(2 T0^2)),
    FWHM = 2 sqrt(ln 2) T0."""
    if kind == "sech":
        t0 = fwhm / (2.0 * math.acosh(math.sqrt(2.0)))
        return 1.0 / np.cosh(t / t0)
    if kind == "gaussian":
        t0 = fwhm / (2.0 * math.sqrt(math.log(2.0)))
        return np.exp(-(t * t) / (2.0 * t0 * t0))
    raise ValueError(kind)


def launch_field(num_modes: int, nt: int, dt: float, kind: str, fwhm: float,
                 energy: float, seed: int) -> np.ndarray:
    """A_p(0, t_k) = w_p sqrt(P0) f(t_k), with P0 chosen so that
    dt * sum_{p,k} |A_p(t_k)|^2 equals the pulse energy."""
    t = time_grid(nt, dt)
    f = pulse_shape(kind, t, fwhm)
    w = random_mode_weights(num_modes, seed)
    p0 = energy / (dt * float(np.sum(f * f)))
    return (w[:, None] * math.sqrt(p0)) * f[None, :].astype(np.complex128)


# ----------------------------------------------------------------------------
# Problem bundles
# ----------------------------------------------------------------------------
@dataclass
class Problem:
    """Everything gmmnlse_create and gmmnlse_propagate consume."""
    name: str
    N: int
    Nt: int
    dt: float
    lam0: float
    n2: float
    beta: np.ndarray          # [N][Nt] rad/m, FFT order, mode-1 frame
    SK: np.ndarray            # [N][N][N][N] 1/m^2
    SR: np.ndarray            # [N][N][N][N] 1/m^2
    fR: float
    hR: np.ndarray            # [Nt] 1/s, t_k = k dt
    self_steepening: int
    A0: np.ndarray            # [N][Nt] complex sqrt(W), t_k = (k - Nt/2) dt
    L: float
    dz: float
    M: int
    tol: float
    extra: dict = field(default_factory=dict)

    @property
    def omega0(self):
        return 2 * np.pi * C_LIGHT / self.lam0


def grin_problem(name, N, Nt, dt, kind, fwhm, energy, L, dz, M, tol, seed,
                 fR=0.0, self_steepening=1, radius=25e-6, na=0.2, lam0=1030e-9,
                 n2=2.3e-20, tau1=12.2e-15, tau2=32e-15, s_from="grid", npts=128):
    modes = grin_mode_indices(N)
    omega0 = 2 * np.pi * C_LIGHT / lam0
    coeffs = []
    for (mx, ny) in modes:
        g = mx + ny
        coeffs.append(taylor_coefficients(
            lambda om, g=g: grin_beta_closed_form(om, g, radius, na), omega0))
    beta = beta_from_taylor(coeffs, omega_grid(Nt, dt))
    w = grin_mode_width(radius, na, lam0)
    if s_from == "grid":
        S = grin_S_grid(modes, w, radius, npts=npts)
    else:
        S = grin_S_gauss_hermite(modes, w)
    hR = raman_response(Nt, dt, tau1, tau2)
    A0 = launch_field(N, Nt, dt, kind, fwhm, energy, seed)
    return Problem(name=name, N=N, Nt=Nt, dt=dt, lam0=lam0, n2=n2, beta=beta,
                   SK=S, SR=S, fR=fR, hR=hR, self_steepening=self_steepening,
                   A0=A0, L=L, dz=dz, M=M, tol=tol,
                   extra=dict(modes=modes, w=w, coeffs=coeffs, seed=seed))


def step_index_problem(name, N, Nt, dt, kind, fwhm, energy, L, dz, M, tol, seed,
                       fR=0.18, self_steepening=1, radius=25e-6, na=0.22,
                       lam0=1030e-9, n2=2.3e-20, npts=400, extent=1.5, overlap=None):
    """`overlap(F, dA) -> S` computes Eq. 2 from the [N][G] grid profiles (for
    instance on the GPU); by default the numpy sums of
    overlap_tensor_from_profiles."""
    modes, info = step_index_modes(radius, na, lam0, N)
    coeffs = step_index_beta_coeffs(radius, na, lam0, modes)
    beta = beta_from_taylor(coeffs, omega_grid(Nt, dt))
    x = (np.arange(npts) - npts / 2 + 0.5) * (2 * extent * radius / npts)
    X, Y = np.meshgrid(x, x, indexing="ij")
    F = np.array([step_index_profile(m, radius, X, Y).ravel() for m in modes])
    S = (overlap or overlap_tensor_from_profiles)(F, (x[1] - x[0]) ** 2)
    S = 0.5 * (S + S.transpose(1, 0, 2, 3))  # symmetrise matmul rounding
    hR = raman_response(Nt, dt)
    A0 = launch_field(N, Nt, dt, kind, fwhm, energy, seed)
    return Problem(name=name, N=N, Nt=Nt, dt=dt, lam0=lam0, n2=n2, beta=beta,
                   SK=S, SR=S, fR=fR, hR=hR, self_steepening=self_steepening,
                   A0=A0, L=L, dz=dz, M=M, tol=tol,
                   extra=dict(modes=modes, info=info, coeffs=coeffs, seed=seed))


def workload(name: str, **over) -> Problem:
    """The named workloads C1..C4, each described by its sizes below (the
    served mix C5 comes from serving_requests).  Keyword overrides change any
    grin_problem argument (e.g. a shorter fiber L for a prefix run)."""
    if name == "C1":  # FP64 Kerr only, N=3, Nt=2^10 over 5 ps
        kw = dict(N=3, Nt=1024, dt=5e-12 / 1024, kind="sech", fwhm=100e-15, energy=10e-9,
                  L=0.05, dz=0.5e-3, M=5, tol=1e-12, seed=1, fR=0.0)
        kw.update(over)
        return grin_problem("C1", **kw)
    if name == "C2":  # Kerr + Raman, N=6, Nt=2^13 over 10 ps
        kw = dict(N=6, Nt=8192, dt=10e-12 / 8192, kind="gaussian", fwhm=200e-15, energy=50e-9,
                  L=0.5, dz=25e-6, M=10, tol=1e-8, seed=2, fR=0.18)
        kw.update(over)
        return grin_problem("C2", **kw)
    if name == "C3":  # N=15 (mode groups 0-4), Nt=2^14 over 20 ps
        kw = dict(N=15, Nt=16384, dt=20e-12 / 16384, kind="gaussian", fwhm=500e-15,
                  energy=200e-9, L=1.0, dz=12.5e-6, M=20, tol=1e-6, seed=3, fR=0.18)
        kw.update(over)
        return grin_problem("C3", **kw)
    if name == "C4":  # step-index, 42 LP modes, Nt=2^13 over 10 ps
        kw = dict(N=42, Nt=8192, dt=10e-12 / 8192, kind="gaussian", fwhm=100e-15,
                  energy=100e-9, L=0.3, dz=37.5e-6, M=16, tol=1e-6, seed=4, fR=0.18)
        kw.update(over)
        return step_index_problem("C4", **kw)
    raise ValueError(name)
