"""Plain FP64 CPU statement of the GMMNLSE and its massively parallel algorithm.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Slow on purpose: every
function follows the paper's formula directly, with numpy's FFT and matrix
product as the only library primitives.  It never uses the symmetry rewrite
that the CUDA path relies on (pair products U_mn, 2 Re terms), so parity
against it checks that rewrite.

Conventions (readings of the paper, each pinned by a test):
  * Fourier sign.  The dispersion operator is written with (i d/dt)^n and the
    self-steepening factor becomes (1 + omega/omega0) in the frequency domain
    (Sec. III.D, definition of D(t) and Eq. MPA_eq); both hold for fields
    varying as exp(-i omega t).  Hence F{f}(omega_q) = sum_k f_k exp(+i omega_q t_k)
    (numpy: Nt * ifft) and F^-1 = fft / Nt, so D_omega = i beta_p(omega).
  * Raman integral of Eq. 1: a causal convolution (h_R * A_m A_n^*)(t) =
    int_0^inf h_R(tau) A_m(t - tau) A_n^*(t - tau) dtau, made circular over
    the time window: dt * sum_k' h[k'] q[(k - k') mod Nt].
  * MPA (Sec. III.D): psi_j = psi_0 + (dz/2) sum_{k=1..j} (I_{k-1} + I_k) with
    I_j = i (n2 w0/c) s(w) F{NL(A_j)} exp(-i beta (z_j - z_0)),
    A_j = F^-1{psi_j exp(+i beta (z_j - z_0))}; initial guess psi_j = psi_0;
    I_0 is evaluated once per long step from the known A(z_0).
  * Convergence measure (the paper only says "a given threshold"):
    eps = ||psi^(n+1) - psi^(n)||_2 / ||psi^(n+1)||_2 over j = 1..M, all modes
    and frequencies.  At least one update is always made.
"""
from __future__ import annotations

import math

import numpy as np

C_LIGHT = 299792458.0

OK = 0
E_NOT_CONVERGED = -4
E_NONFINITE = -5


# ----------------------------------------------------------------------------
# Fourier transforms (Sec. III.D, Eq. cov)
# ----------------------------------------------------------------------------
def freq_from_time(a):
    """F{a}(omega_q) = sum_k a_k exp(+i omega_q t_k), omega_q in FFT order."""
    a = np.asarray(a)
    return np.fft.ifft(a, axis=-1) * a.shape[-1]


def time_from_freq(af):
    """Inverse of freq_from_time: a_k = (1/Nt) sum_q af_q exp(-i omega_q t_k)."""
    af = np.asarray(af)
    return np.fft.fft(af, axis=-1) / af.shape[-1]


# ----------------------------------------------------------------------------
# Fiber description
# ----------------------------------------------------------------------------
def _coupling_tensor(S):
    """A coupling tensor as given: complex128 if it has complex entries,
    else float64."""
    S = np.asarray(S)
    return S.astype(np.complex128) if np.iscomplexobj(S) else S.astype(np.float64)


class Fiber:
    """The inputs of Eq. 1: per-mode beta_p(omega) [N][Nt] (rad/m, FFT order,
    mode-1 frame), coupling tensors S^K, S^R [N]^4 (1/m^2), Raman fraction f_R,
    Raman response h_R [Nt] sampled at t_k = k dt (1/s), time step dt (s),
    centre wavelength lam0 (m), n2 (m^2/W) and the self-steepening switch."""

    def __init__(self, beta, SK, SR, fR, hR, dt, lam0, n2, self_steepening=True, Q=None, gain=None,
                 Q_profile=None, Q_profile_dz=None, sat=0.0):
        self.beta = np.asarray(beta, dtype=np.float64)
        # linear mode coupling Q[n][p] (Sec. IV, "Linear mode coupling"): the
        # extra right-hand-side term C_p = i sum_n Q_np A_n, or None
        self.Q = None if Q is None else np.asarray(Q, dtype=np.float64)
        # its longitudinal profile (Sec. IV: [n^2 - n_p^2] = eps(x, y) f(z)):
        # Q_np(z) = Q_np f(z), f sampled at z = k Q_profile_dz and linearly
        # interpolated (None: f = 1)
        self.Q_profile = None if Q_profile is None else np.asarray(Q_profile, dtype=np.float64)
        self.Q_profile_dz = Q_profile_dz
        # small-signal field gain g_p [1/m] (Sec. IV, "Saturating gain", its
        # lowest order): the extra term g_p A_p, or None
        self.gain = None if gain is None else np.asarray(gain, dtype=np.float64)
        # its saturation (the same passage's first-order term):
        # - sat sum_{l,m,n} S^R_plmn A_l int A_m A_n^* dtau, sat = 1/I_sat of
        # the paper's expression (0: none)
        self.sat = float(sat)
        self.N, self.Nt = self.beta.shape
        # S^K, S^R: real for one linear polarization and real mode profiles
        # (Eq. 2), complex in general (Eq. 1 with complex or vector mode
        # fields; no symmetry assumed)
        self.SK = _coupling_tensor(SK)
        self.SR = None if SR is None else _coupling_tensor(SR)
        self.fR = float(fR)
        self.hR = None if hR is None else np.asarray(hR, dtype=np.float64)
        self.dt = float(dt)
        self.lam0 = float(lam0)
        self.n2 = float(n2)
        self.self_steepening = bool(self_steepening)
        self.omega = 2.0 * np.pi * np.fft.fftfreq(self.Nt, d=self.dt)
        self.omega0 = 2.0 * np.pi * C_LIGHT / self.lam0
        # i (n2 omega0 / c) (1 + omega/omega0): Eq. MPA_eq prefactor
        self.gamma0 = self.n2 * self.omega0 / C_LIGHT
        self.shock = (1.0 + self.omega / self.omega0) if self.self_steepening \
            else np.ones(self.Nt)

    @classmethod
    def from_problem(cls, prob, **over):
        kw = dict(beta=prob.beta, SK=prob.SK, SR=prob.SR, fR=prob.fR, hR=prob.hR,
                  dt=prob.dt, lam0=prob.lam0, n2=prob.n2,
                  self_steepening=prob.self_steepening)
        kw.update(over)
        return cls(**kw)


# ----------------------------------------------------------------------------
# Nonlinear bracket of Eq. 1
# ----------------------------------------------------------------------------
def circular_convolution(h, q, dt):
    """(h * q)_k = dt sum_k' h[k'] q[(k - k') mod Nt], by the convolution
    theorem (numpy FFT).  q: [..., Nt]."""
    return dt * np.fft.ifft(np.fft.fft(h) * np.fft.fft(q, axis=-1), axis=-1)


def circular_convolution_direct(h, q, dt):
    """The same sum written out, O(Nt^2); for small Nt only."""
    h = np.asarray(h)
    q = np.asarray(q)
    nt = h.shape[-1]
    out = np.zeros(q.shape, dtype=np.complex128)
    for k in range(nt):
        acc = 0.0
        for kp in range(nt):
            acc = acc + h[kp] * q[..., (k - kp) % nt]
        out[..., k] = dt * acc
    return out


def _pair_products(A):
    """Q[m, n, t] = A_m(t) A_n^*(t)."""
    return A[:, None, :] * np.conj(A)[None, :, :]


def kerr_sum(SK, A):
    """sum_{l,m,n} S^K_plmn A_l A_m A_n^*  (Eq. 1, Kerr bracket), as
    sum_l A_l (sum_{m,n} S^K_plmn A_m A_n^*).  A: [N][Nt] -> [N][Nt]."""
    N = A.shape[0]
    Q = _pair_products(A).reshape(N * N, -1)
    T = (np.asarray(SK).reshape(N * N, N * N) @ Q).reshape(N, N, -1)  # T[p,l,t]
    return np.einsum("plt,lt->pt", T, A)


def raman_sum(SR, A, hR, dt):
    """sum_{l,m,n} S^R_plmn A_l (h_R * A_m A_n^*)  (Eq. 1, Raman bracket)."""
    N = A.shape[0]
    H = circular_convolution(hR, _pair_products(A), dt).reshape(N * N, -1)
    T = (np.asarray(SR).reshape(N * N, N * N) @ H).reshape(N, N, -1)
    return np.einsum("plt,lt->pt", T, A)


def nonlinear_bracket(fib: Fiber, A):
    """(1 - f_R) Kerr + f_R Raman, the bracket of Eq. 1, in the time domain."""
    out = (1.0 - fib.fR) * kerr_sum(fib.SK, A)
    if fib.fR != 0.0:
        out = out + fib.fR * raman_sum(fib.SR, A, fib.hR, fib.dt)
    return out


def coupling_factor(fib: Fiber, z):
    """f(z) of the coupling profile Q_np(z) = Q_np f(z): linear interpolation
    of the samples f_k at z = k dz_f (held constant past the last sample)."""
    if fib.Q_profile is None:
        return 1.0
    zs = np.arange(len(fib.Q_profile)) * fib.Q_profile_dz
    return float(np.interp(z, zs, fib.Q_profile))


def saturation_term(fib: Fiber, A):
    """sum_{l,m,n} S^R_plmn A_l(t) int A_m(tau) A_n^*(tau) dtau (the
    saturating-gain term of Sec. IV without its factor -1/I_sat), the
    integral as the sum dt sum_k over the time window.  A: [N][Nt] time
    domain -> [N][Nt]."""
    N = A.shape[0]
    SR = fib.SK if fib.SR is None else fib.SR
    E = fib.dt * (A @ np.conj(A).T)  # E[m, n] = int A_m A_n^* dtau
    T = (np.asarray(SR).reshape(N * N, N * N) @ E.reshape(N * N)).reshape(N, N)  # T[p, l]
    return T @ A


def nonlinear_operator(fib: Fiber, Aw, z=0.0):
    """N(A~) = i (n2 w0/c) s(w) F{bracket(F^-1 A~)} for a spectral field A~ at
    fiber position z, plus the terms Sec. IV adds to the right-hand side of
    Eq. 1 when the fiber has them: the linear mode coupling
    C_p = i sum_n Q_np(z) A~_n, the small-signal gain g_p A~_p and its
    saturation - sat F{sum_lmn S^R_plmn A_l int A_m A_n^* dtau}."""
    At = time_from_freq(Aw)
    NL = nonlinear_bracket(fib, At)
    out = 1j * fib.gamma0 * fib.shock * freq_from_time(NL)
    if fib.Q is not None:
        out = out + 1j * coupling_factor(fib, z) * (fib.Q.T @ Aw)  # (Q^T A)_p = sum_n Q[n][p] A_n
    if fib.gain is not None:
        out = out + fib.gain[:, None] * Aw
    if fib.sat != 0.0:
        out = out - fib.sat * freq_from_time(saturation_term(fib, At))
    return out


# ----------------------------------------------------------------------------
# MPA (Sec. III.D)
# ----------------------------------------------------------------------------
def phase_factor(fib: Fiber, zrel):
    """exp(D_omega (z - z0)) = exp(i beta_p(omega) (z - z0)), FP64.  The
    argument beta * (z - z0) is formed in FP64 and reduced mod 2 pi by the
    C library's sin/cos."""
    return np.exp(1j * (fib.beta * zrel))


def integrand(fib: Fiber, psi_j, zrel, z0=0.0):
    """Integrand of Eq. MPA_eq at z_j = z0 + zrel: A_j = F^-1{psi_j e^{D (z_j - z0)}},
    I_j = i (n2 w0/c) s(w) F{NL(A_j)} e^{-D (z_j - z0)}."""
    E = phase_factor(fib, zrel)
    return nonlinear_operator(fib, psi_j * E, z0 + zrel) * np.conj(E)


def mpa_long_step(fib: Fiber, psi0, dz, M, tol, max_iter=50, fixed_iters=0, z0=0.0):
    """One long step L = M dz from z0 (Sec. III.D).  psi0 = A~(z0, omega).

    Returns (A~(z0 + L), iterations, eps trace, status).  Iteration n builds
    psi^(n+1) from the integrands of psi^(n) by the trapezoid rule over z';
    it stops when eps < tol (or after fixed_iters updates when that is > 0);
    status E_NOT_CONVERGED after max_iter updates, E_NONFINITE on NaN/Inf."""
    zrel = [j * dz for j in range(M + 1)]
    I = [None] * (M + 1)
    I[0] = integrand(fib, psi0, zrel[0], z0)
    psi = [psi0] * (M + 1)  # psi^(1)(z_j) = psi(z0)
    trace = []
    n = 0
    status = OK
    while True:
        for j in range(1, M + 1):
            I[j] = integrand(fib, psi[j], zrel[j], z0)
        new = [psi0]
        acc = np.zeros_like(psi0)
        for j in range(1, M + 1):
            acc = acc + 0.5 * dz * (I[j - 1] + I[j])
            new.append(psi0 + acc)
        diff = sum(float(np.sum(np.abs(new[j] - psi[j]) ** 2)) for j in range(1, M + 1))
        size = sum(float(np.sum(np.abs(new[j]) ** 2)) for j in range(1, M + 1))
        finite = math.isfinite(diff) and math.isfinite(size)
        eps = math.sqrt(diff / size) if (finite and size > 0) else (0.0 if finite else math.nan)
        psi = new
        n += 1
        trace.append(eps)
        if not finite:
            status = E_NONFINITE
            break
        if fixed_iters > 0:
            if n >= fixed_iters:
                break
            continue
        if eps < tol:
            break
        if n >= max_iter:
            status = E_NOT_CONVERGED
            break
    return psi[M] * phase_factor(fib, zrel[M]), n, trace, status


def substep_schedule(L, dz, M):
    """Long-step sizes for a fiber of length L: round(L/dz) substeps of dz in
    long steps of M, the last one shorter if M does not divide the count."""
    total = int(round(L / dz))
    if total < 1 or abs(total * dz - L) > 1e-9 * max(L, dz):
        raise ValueError("L must be a positive whole number of dz")
    sizes = [M] * (total // M)
    if total % M:
        sizes.append(total % M)
    return sizes


def mpa_propagate(fib: Fiber, A0, L, dz, M, tol, max_iter=50, fixed_iters=0):
    """Propagate A0 (time domain [N][Nt]) over a fiber of length L with the
    MPA.  Returns (A(L) in the time domain, stats dict).  On failure the field
    is the one at the last completed long step and stats['z'] says where."""
    psi = freq_from_time(np.asarray(A0, dtype=np.complex128))
    stats = dict(iters=[], eps=[], z=0.0, status=OK)
    done = 0
    for Mj in substep_schedule(L, dz, M):
        out, n, trace, status = mpa_long_step(fib, psi, dz, Mj, tol, max_iter, fixed_iters, z0=done * dz)
        stats["iters"].append(n)
        stats["eps"].append(trace)
        if status != OK:
            stats["status"] = status
            break
        psi = out
        done += Mj
    stats["z"] = done * dz
    return time_from_freq(psi), stats


# ----------------------------------------------------------------------------
# Comparators used as pins
# ----------------------------------------------------------------------------
def iptrap_propagate(fib: Fiber, A0, L, dz, tol=1e-15, max_iter=200):
    """Sequential interaction-picture trapezoid rule, one dz at a time:
    A_j = e^{D dz}(A_{j-1} + (dz/2) N(A_{j-1})) + (dz/2) N(A_j), each step
    solved by fixed-point iteration until the update stops shrinking."""
    Aw = freq_from_time(np.asarray(A0, dtype=np.complex128))
    E1 = phase_factor(fib, dz)
    steps = int(round(L / dz))
    for k in range(steps):
        z = k * dz
        base = E1 * (Aw + 0.5 * dz * nonlinear_operator(fib, Aw, z))
        X = base + 0.5 * dz * E1 * nonlinear_operator(fib, Aw, z)
        prev = np.inf
        for _ in range(max_iter):
            Xn = base + 0.5 * dz * nonlinear_operator(fib, X, z + dz)
            d = float(np.linalg.norm(Xn - X)) / max(float(np.linalg.norm(Xn)), 1e-300)
            X = Xn
            if d < tol or d >= prev:
                break
            prev = d
        Aw = X
    return time_from_freq(Aw)


def rk4ip_propagate(fib: Fiber, A0, L, h):
    """Fourth-order Runge-Kutta in the interaction picture (Hult, J. Lightwave
    Technol. 25, 3770, 2007) with half-step dispersion exp(D h/2)."""
    Aw = freq_from_time(np.asarray(A0, dtype=np.complex128))
    Eh = phase_factor(fib, 0.5 * h)
    steps = int(round(L / h))
    Nop = lambda X, z: nonlinear_operator(fib, X, z)  # noqa: E731
    for k in range(steps):
        z = k * h  # the stages sit at z, z + h/2, z + h/2, z + h
        AI = Eh * Aw
        k1 = Eh * Nop(Aw, z)
        k2 = Nop(AI + 0.5 * h * k1, z + 0.5 * h)
        k3 = Nop(AI + 0.5 * h * k2, z + 0.5 * h)
        k4 = Nop(Eh * (AI + h * k3), z + h)
        Aw = Eh * (AI + (h / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3)) + (h / 6.0) * k4
    return time_from_freq(Aw)


# ----------------------------------------------------------------------------
# Mode overlap tensor (Eq. 2)
# ----------------------------------------------------------------------------
def overlap_tensor(F, dA):
    """S_plmn = int F_p F_l F_m F_n dA / sqrt(int F_p^2 dA int F_l^2 dA
    int F_m^2 dA int F_n^2 dA) (Eq. 2) for real profiles F [N][G] sampled on
    G grid cells of area dA: the integrals as plain sums over the cells."""
    F = np.asarray(F, dtype=np.float64)
    norm = np.sum(F * F, axis=1) * dA
    quad = np.einsum("pg,lg,mg,ng->plmn", F, F, F, F) * dA
    den = np.sqrt(np.einsum("p,l,m,n->plmn", norm, norm, norm, norm))
    return quad / den


# ----------------------------------------------------------------------------
# Invariants
# ----------------------------------------------------------------------------
def energy_spectral(Aw):
    """sum_p sum_q |A~_p(omega_q)|^2 (proportional to the pulse energy)."""
    return float(np.sum(np.abs(Aw) ** 2))


def photon_number(fib: Fiber, Aw):
    """sum_p sum_q |A~_p|^2 / (omega0 + omega_q) over bins with omega0 +
    omega_q > 0 (proportional to the photon number)."""
    w = fib.omega0 + fib.omega
    mask = w > 0
    return float(np.sum(np.abs(Aw[:, mask]) ** 2 / w[None, mask]))


# ----------------------------------------------------------------------------
# Length scales of the step sizes (Sec. III.D)
# ----------------------------------------------------------------------------
def length_scales(fib: Fiber, A0):
    """The two length scales that set the MPA's step sizes (Sec. III.D):
    the nonlinear length z_NL = 1 / (gamma0 S_max P0), the single-mode
    estimate A_eff/(n2 omega0 P0) with 1/A_eff the largest self-overlap
    |S^K_pppp| and the speed of light that the paper's printed form omits
    (gamma0 = n2 omega0 / c), P0 the peak of sum_p |A_p(t)|^2; and the
    intermode beat length z_IM = 1 / max_p |delta beta0^(p)|, delta beta0^(p)
    = beta_p(omega = 0) - beta_1(omega = 0) (infinite for a single mode).
    A0: [N][Nt] time domain.  Returns (z_NL, z_IM)."""
    A0 = np.asarray(A0)
    P0 = float(np.max(np.sum(np.abs(A0) ** 2, axis=0)))
    S_max = max(abs(complex(fib.SK[p, p, p, p])) for p in range(fib.N))
    z_nl = 1.0 / (fib.gamma0 * S_max * P0)
    db0 = np.abs(fib.beta[:, 0] - fib.beta[0, 0])
    z_im = 1.0 / float(np.max(db0)) if np.max(db0) > 0 else math.inf
    return z_nl, z_im
