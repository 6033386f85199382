"""FP64 CPU oracle for the explicit forward-Euler phase-field / reaction-diffusion step.

TEST INFRASTRUCTURE ONLY.  This package is imported by ``tests/``, by
``__graft_entry__.smoke()`` and by the CPU-baseline / reference arm of ``bench.py``, and by
nothing else.  It shares no code with the CUDA library and never calls it; the CUDA path
never imports it.

Every function is plain numpy in float64 and follows the paper's definitions directly:

* grid layout: row-major with x fastest (Sec. 2.2.1 "Uniform Grid"); periodic sides
  (the driver example, Fig. "driver_implementation" in Sec. 2.4, sets every edge
  periodic), done here with ``np.roll``;
* the second-order central Laplacian, 5 points in 2D and 7 points in 3D
  (Sec. 2.2.2 "Finite Difference Stencils");
* Model A (Allen-Cahn) and Model B (Cahn-Hilliard) equations of motion (Sec. 3,
  the first two numbered equations), with the coefficient names of the model
  definitions figure (Fig. "models_abc_definitions"): A uses c1 (linear) and c2 (cubic);
  B uses c1, c2 and a mobility M multiplying the whole right-hand side;
* Model C (eutectic; Sec. 3, third numbered equation and its model definition): a
  non-conserved psi and a conserved m coupled through c5,
  dpsi/dt = lap psi + c1 psi - c2 psi^3 + 2 c5 psi m,
  dm/dt = lap(c4 m^3 - c3 m - c5 psi^2 - lap m);
* Gray-Scott, which the paper names as a reaction-diffusion example (Sec. 1) but does not
  write out, in its standard two-species form
  du/dt = Du lap u - u v^2 + F (1 - u),  dv/dt = Dv lap v + u v^2 - (F + k) v;
* N coupled species (any number of fields, Sec. 2.3) of reaction-diffusion type,
  du_i/dt = D_i lap u_i + sum_m K[i][m] prod_j u_j^E[m][j], polynomial rates;
* the forward-Euler solver (Sec. 2.4.1): x^{n+1} = x^n + dt f(x^n), every field updated
  from the same x^n, i.e. the paper's ``equation()`` then ``step()`` split (Sec. 2.2.4);
* the discrete free energy whose gradient flow Model A is, and the discrete adjoint of
  the Gray-Scott forward-Euler map (reverse-mode derivative of the time loop).

Parity status: every function here is pinned by the tests in ``tests/test_oracle_*.py``
(closed forms, brute force on tiny grids, invariants, complex-step derivatives).
"""
from __future__ import annotations

import itertools

import numpy as np

MODELS = ("ac", "ch", "gs", "c", "rd")


def _f64(x):
    a = np.asarray(x)
    if np.iscomplexobj(a):
        return a.astype(np.complex128)
    return a.astype(np.float64)


# ------------------------------------------------------------------ stencils (Sec. 2.2.2)

def laplacian(phi, h: float = 1.0):
    """Periodic second-order Laplacian: sum over axes of (phi[+1] + phi[-1] - 2 phi) / h^2.

    5-point in 2D, 7-point in 3D (3-point in 1D).  Works for real or complex arrays.
    """
    phi = _f64(phi)
    out = np.zeros_like(phi)
    for ax in range(phi.ndim):
        out += (np.roll(phi, 1, axis=ax) - phi) + (np.roll(phi, -1, axis=ax) - phi)
    return out / (h * h)


# Further Laplacian stencils of Sec. 2.2.2 (second-order isotropic 9-point in 2D and
# 19- and 27-point in 3D; fourth-order 9-point in 2D), written from their weights:
#   "9iso":  (1/6h^2) [4 (axial neighbours) + (diagonal neighbours) - 20 phi]
#   "9o4":   (1/12h^2) sum over axes [16 (phi[+1] + phi[-1]) - (phi[+2] + phi[-2]) - 30 phi]
#   "19iso": (1/6h^2) [2 (face neighbours) + (edge neighbours) - 24 phi]
#   "27iso": (1/30h^2) [14 (face neighbours) + 3 (edge neighbours) + (corner neighbours)
#            - 128 phi]
# "std" is the 5-point (2D) / 7-point (3D) stencil above.
STENCILS_2D = ("std", "9iso", "9o4")
STENCILS_3D = ("std", "19iso", "27iso")


def laplacian_stencil(phi, h: float = 1.0, stencil: str = "std"):
    """Periodic Laplacian with the named stencil."""
    phi = _f64(phi)
    if stencil == "std":
        return laplacian(phi, h)
    d = phi.ndim
    sh = lambda a, *o: np.roll(a, tuple(-x for x in o), axis=tuple(range(len(o))))  # a[x + o]
    if stencil == "9iso" and d == 2:
        axial = sh(phi, 1, 0) + sh(phi, -1, 0) + sh(phi, 0, 1) + sh(phi, 0, -1)
        diag = sh(phi, 1, 1) + sh(phi, 1, -1) + sh(phi, -1, 1) + sh(phi, -1, -1)
        return (4.0 * axial + diag - 20.0 * phi) / (6.0 * h * h)
    if stencil == "9o4" and d == 2:
        out = np.zeros_like(phi)
        for ax in range(2):
            p1 = np.roll(phi, 1, axis=ax) + np.roll(phi, -1, axis=ax)
            p2 = np.roll(phi, 2, axis=ax) + np.roll(phi, -2, axis=ax)
            out += 16.0 * p1 - p2 - 30.0 * phi
        return out / (12.0 * h * h)
    if stencil == "19iso" and d == 3:
        faces = np.zeros_like(phi)
        edges = np.zeros_like(phi)
        for ax in range(3):
            faces += np.roll(phi, 1, axis=ax) + np.roll(phi, -1, axis=ax)
        for a in range(3):
            for b in range(a + 1, 3):
                for sa in (1, -1):
                    for sb in (1, -1):
                        edges += np.roll(np.roll(phi, sa, axis=a), sb, axis=b)
        return (2.0 * faces + edges - 24.0 * phi) / (6.0 * h * h)
    if stencil == "27iso" and d == 3:
        faces = np.zeros_like(phi)
        edges = np.zeros_like(phi)
        corners = np.zeros_like(phi)
        for o in itertools.product((-1, 0, 1), repeat=3):
            nz = sum(1 for x in o if x != 0)
            if nz == 1:
                faces += sh(phi, *o)
            elif nz == 2:
                edges += sh(phi, *o)
            elif nz == 3:
                corners += sh(phi, *o)
        return (14.0 * faces + 3.0 * edges + corners - 128.0 * phi) / (30.0 * h * h)
    raise ValueError(f"stencil {stencil!r} is not defined for {d}D")


# ------------------------------------------------------------ right-hand sides (Sec. 3)

def rhs_allen_cahn(phi, c1: float = 1.0, c2: float = 1.0, h: float = 1.0, stencil="std"):
    """Model A: dphi/dt = lap phi + c1 phi - c2 phi^3."""
    phi = _f64(phi)
    return laplacian_stencil(phi, h, stencil) + c1 * phi - c2 * phi ** 3


def chemical_potential(phi, c1: float = 1.0, c2: float = 1.0, h: float = 1.0, stencil="std"):
    """Model B chemical potential mu = c2 phi^3 - c1 phi - lap phi."""
    phi = _f64(phi)
    return c2 * phi ** 3 - c1 * phi - laplacian_stencil(phi, h, stencil)


def rhs_cahn_hilliard(phi, c1: float = 1.0, c2: float = 1.0, M: float = 1.0, h: float = 1.0,
                      stencil="std"):
    """Model B: dphi/dt = M lap mu = -M lap^2 phi - M lap (c1 phi - c2 phi^3)."""
    return M * laplacian_stencil(chemical_potential(phi, c1, c2, h, stencil), h, stencil)


def rhs_gray_scott(u, v, Du: float, Dv: float, F: float, k: float, h: float = 1.0,
                   stencil="std"):
    """Gray-Scott: (Du lap u - u v^2 + F (1-u),  Dv lap v + u v^2 - (F+k) v)."""
    u = _f64(u)
    v = _f64(v)
    uvv = u * v * v
    fu = Du * laplacian_stencil(u, h, stencil) - uvv + F * (1.0 - u)
    fv = Dv * laplacian_stencil(v, h, stencil) + uvv - (F + k) * v
    return fu, fv


def rhs_model_c(psi, m, c1=1.0, c2=1.0, c3=1.0, c4=1.0, c5=1.0, h: float = 1.0,
                stencil="std"):
    """Model C: (lap psi + c1 psi - c2 psi^3 + 2 c5 psi m,
                 lap(c4 m^3 - c3 m - c5 psi^2 - lap m))."""
    psi = _f64(psi)
    m = _f64(m)
    lap = lambda a: laplacian_stencil(a, h, stencil)
    f_psi = lap(psi) + c1 * psi - c2 * psi ** 3 + 2.0 * c5 * psi * m
    mu_m = c4 * m ** 3 - c3 * m - c5 * psi ** 2 - lap(m)
    return f_psi, lap(mu_m)


# ---------------------------------------- N coupled species (reaction-diffusion, generic)
#
# The paper writes a model as a set of coupled equations of motion over any number of fields
# (Sec. 2.3); Gray-Scott (Sec. 1) is the two-species reaction-diffusion case. The generic
# family here couples N fields through polynomial reaction terms:
#   du_i/dt = D_i lap u_i + sum_m K[i][m] prod_j u_j ** E[m][j]
# with M monomials whose integer exponents E[m][j] are in 0..3, and rates K. Coefficient
# layout (the C interface's): D_0 .. D_{N-1}, M, then E row by row (M rows of N), then K row by
# row (N rows of M).

RD_MAX_FIELDS = 4
RD_MAX_MONOMIALS = 8


def rd_unpack(coeffs, n_fields: int):
    """(D, E, K) from the flat coefficient list of an N-species system."""
    c = [float(x) for x in coeffs]
    N = int(n_fields)
    if not 1 <= N <= RD_MAX_FIELDS or len(c) < N + 1:
        raise ValueError("bad field count or coefficient list")
    D = np.array(c[:N])
    M = int(round(c[N]))
    if c[N] != M or not 0 <= M <= RD_MAX_MONOMIALS or len(c) != N + 1 + 2 * N * M:
        raise ValueError("bad monomial count or coefficient list length")
    E = np.array(c[N + 1:N + 1 + M * N]).reshape(M, N)
    if not np.all((E == np.round(E)) & (E >= 0) & (E <= 3)):
        raise ValueError("exponents must be integers in 0..3")
    K = np.array(c[N + 1 + M * N:]).reshape(N, M)
    return D, E.astype(int), K


def rd_pack(D, E, K):
    """The flat coefficient list of (D, E, K)."""
    D = [float(x) for x in D]
    E = np.asarray(E, dtype=float).reshape(-1, len(D))
    K = np.asarray(K, dtype=float).reshape(len(D), E.shape[0])
    return tuple(D) + (float(E.shape[0]),) + tuple(E.ravel()) + tuple(K.ravel())


def rhs_rd(fields, coeffs, h: float = 1.0, stencil: str = "std"):
    """N-species reaction-diffusion right-hand side (one array per field)."""
    u = [_f64(f) for f in fields]
    D, E, K = rd_unpack(coeffs, len(u))
    mono = []
    for row in E:
        p = np.ones_like(u[0])
        for j, e in enumerate(row):
            p = p * u[j] ** int(e)
        mono.append(p)
    out = []
    for i in range(len(u)):
        f = D[i] * laplacian_stencil(u[i], h, stencil)
        for mm, p in enumerate(mono):
            f = f + K[i, mm] * p
        out.append(f)
    return tuple(out)


def rhs(model: str, fields, coeffs, h: float = 1.0, stencil: str = "std"):
    """Right-hand side f(x) of ``model`` for the tuple of fields ``x``."""
    if model == "rd":
        return rhs_rd(fields, coeffs, h, stencil)
    if model == "ac":
        return (rhs_allen_cahn(fields[0], *coeffs, h=h, stencil=stencil),)
    if model == "ch":
        return (rhs_cahn_hilliard(fields[0], *coeffs, h=h, stencil=stencil),)
    if model == "gs":
        return rhs_gray_scott(fields[0], fields[1], *coeffs, h=h, stencil=stencil)
    if model == "c":
        return rhs_model_c(fields[0], fields[1], *coeffs, h=h, stencil=stencil)
    raise ValueError(f"unknown model {model!r}")


# ----------------------------------------------------------- forward Euler (Sec. 2.4.1)

def euler_step(model: str, fields, coeffs, dt: float, h: float = 1.0, stencil: str = "std"):
    """One explicit step x^{n+1} = x^n + dt f(x^n); all fields read x^n."""
    fields = tuple(_f64(f) for f in fields)
    f = rhs(model, fields, coeffs, h, stencil)
    return tuple(x + dt * fx for x, fx in zip(fields, f))


def run(model: str, fields, coeffs, dt: float, n_steps: int, h: float = 1.0,
        stencil: str = "std"):
    """``n_steps`` forward-Euler steps from ``fields``."""
    x = tuple(_f64(f) for f in fields)
    for _ in range(int(n_steps)):
        x = euler_step(model, x, coeffs, dt, h, stencil)
    return x


# ------------------------------------------------------------------------ reductions

def mass(phi, h: float = 1.0) -> float:
    """Discrete integral h^d * sum(phi)."""
    phi = _f64(phi)
    return float(h ** phi.ndim * phi.sum())


def energy(phi, c1: float = 1.0, c2: float = 1.0, h: float = 1.0):
    """Discrete free energy E = h^d sum_x [ 1/2 sum_i ((phi_{x+e_i}-phi_x)/h)^2
    - c1/2 phi^2 + c2/4 phi^4 ].

    -dE/dphi_x / h^d equals the Model A right-hand side exactly, so Model A is the discrete
    gradient flow of E and Model B its lap-weighted flow with mu = dE/dphi_x / h^d.
    """
    phi = _f64(phi)
    grad2 = np.zeros_like(phi)
    for ax in range(phi.ndim):
        d = (np.roll(phi, -1, axis=ax) - phi) / h
        grad2 += d * d
    dens = 0.5 * grad2 - 0.5 * c1 * phi ** 2 + 0.25 * c2 * phi ** 4
    return h ** phi.ndim * dens.sum()


def energy_model_c(psi, m, c1=1.0, c2=1.0, c3=1.0, c4=1.0, c5=1.0, h: float = 1.0):
    """Model C free energy h^d sum_x [ 1/2 |grad psi|^2 - c1/2 psi^2 + c2/4 psi^4
    + 1/2 |grad m|^2 - c3/2 m^2 + c4/4 m^4 - c5 psi^2 m ] (forward differences).

    -dE/dpsi / h^d is the psi right-hand side and dE/dm / h^d the m chemical potential.
    """
    psi = _f64(psi)
    m = _f64(m)
    g = np.zeros(psi.shape, dtype=np.result_type(psi, m))
    for ax in range(psi.ndim):
        dp = (np.roll(psi, -1, axis=ax) - psi) / h
        dm = (np.roll(m, -1, axis=ax) - m) / h
        g += dp * dp + dm * dm
    dens = (0.5 * g - 0.5 * c1 * psi ** 2 + 0.25 * c2 * psi ** 4 - 0.5 * c3 * m ** 2
            + 0.25 * c4 * m ** 4 - c5 * psi ** 2 * m)
    return h ** psi.ndim * dens.sum()


# --------------------------------------------------------- Gray-Scott discrete adjoint

def gray_scott_loss(u, v, u_target, v_target) -> float:
    """L = 1/2 sum over sites of (u - u*)^2 + (v - v*)^2."""
    du = _f64(u) - _f64(u_target)
    dv = _f64(v) - _f64(v_target)
    return 0.5 * float((du * du).sum() + (dv * dv).sum())


def gray_scott_adjoint_step(u, v, a, b, Du, Dv, F, k, dt, h=1.0):
    """Reverse step of the forward-Euler Gray-Scott map x^{n+1} = x^n + dt f(x^n).

    With (u, v) = x^n and (a, b) = lambda^{n+1} = dL/dx^{n+1}, returns lambda^n =
    lambda^{n+1} + dt J(x^n)^T lambda^{n+1} and this step's contribution
    dt (df/dtheta)(x^n)^T lambda^{n+1} to the gradient w.r.t. theta = (Du, Dv, F, k).
    The periodic Laplacian is symmetric, so its transpose is itself.
    """
    u, v, a, b = (_f64(t) for t in (u, v, a, b))
    a_new = a + dt * (Du * laplacian(a, h) - (v * v + F) * a + v * v * b)
    b_new = b + dt * (Dv * laplacian(b, h) - 2.0 * u * v * a + (2.0 * u * v - F - k) * b)
    g = np.array([
        dt * float((a * laplacian(u, h)).sum()),            # d/dDu
        dt * float((b * laplacian(v, h)).sum()),            # d/dDv
        dt * float(((1.0 - u) * a - v * b).sum()),          # d/dF
        -dt * float((v * b).sum()),                          # d/dk
    ])
    return a_new, b_new, g


def gray_scott_adjoint(u0, v0, coeffs, dt, n_steps, dLdu_N, dLdv_N, h=1.0):
    """Gradient of a final-state loss through ``n_steps`` forward-Euler Gray-Scott steps.

    Stores the whole forward trajectory (no checkpointing), then runs the reverse steps
    from n = N-1 down to 0.  Returns (dL/du0, dL/dv0, dL/d(Du, Dv, F, k)).
    """
    Du, Dv, F, k = coeffs
    traj = [(_f64(u0), _f64(v0))]
    for _ in range(int(n_steps)):
        traj.append(euler_step("gs", traj[-1], coeffs, dt, h))
    a, b = _f64(dLdu_N), _f64(dLdv_N)
    g = np.zeros(4)
    for n in range(int(n_steps) - 1, -1, -1):
        u, v = traj[n]
        a, b, gn = gray_scott_adjoint_step(u, v, a, b, Du, Dv, F, k, dt, h)
        g += gn
    return a, b, g


def allen_cahn_adjoint_step(phi, lam, c1, c2, dt, h=1.0):
    """Reverse step of x' = x + dt (lap x + c1 x - c2 x^3) at x = phi^n, lam = lambda^{n+1}:
    lambda^n = lam + dt (lap lam + (c1 - 3 c2 phi^2) lam); gradient terms for (c1, c2)."""
    phi, lam = _f64(phi), _f64(lam)
    lam_new = lam + dt * (laplacian(lam, h) + (c1 - 3.0 * c2 * phi * phi) * lam)
    g = np.array([dt * float((lam * phi).sum()), -dt * float((lam * phi ** 3).sum())])
    return lam_new, g


def cahn_hilliard_adjoint_step(phi, lam, c1, c2, M, dt, h=1.0):
    """Reverse step of x' = x + dt M lap mu(x), mu = c2 x^3 - c1 x - lap x, at x = phi^n:
    with w = lap lam, lambda^n = lam + dt M [(3 c2 phi^2 - c1) w - lap w] (lap symmetric);
    gradient terms for (c1, c2, M)."""
    phi, lam = _f64(phi), _f64(lam)
    w = laplacian(lam, h)
    lam_new = lam + dt * M * ((3.0 * c2 * phi * phi - c1) * w - laplacian(w, h))
    mu = chemical_potential(phi, c1, c2, h)
    g = np.array([-dt * M * float((w * phi).sum()), dt * M * float((w * phi ** 3).sum()),
                  dt * float((w * mu).sum())])
    return lam_new, g


def phase_field_adjoint(model, phi0, coeffs, dt, n_steps, dLdphi_N, h=1.0):
    """dL/dphi0 and dL/dcoeffs of a final-state loss through n forward-Euler steps of Model A
    ("ac", coeffs (c1, c2)) or Model B ("ch", coeffs (c1, c2, M)); stores the trajectory."""
    traj = [_f64(phi0)]
    for _ in range(int(n_steps)):
        traj.append(euler_step(model, (traj[-1],), coeffs, dt, h)[0])
    lam = _f64(dLdphi_N)
    g = np.zeros(len(coeffs))
    for n in range(int(n_steps) - 1, -1, -1):
        if model == "ac":
            lam, gn = allen_cahn_adjoint_step(traj[n], lam, *coeffs, dt, h)
        else:
            lam, gn = cahn_hilliard_adjoint_step(traj[n], lam, *coeffs, dt, h)
        g += gn
    return lam, g


def gray_scott_final_and_loss(u0, v0, coeffs, dt, n_steps, u_target, v_target, h=1.0):
    """Forward run then loss; returns (u_N, v_N, L)."""
    uN, vN = run("gs", (u0, v0), coeffs, dt, n_steps, h)
    return uN, vN, gray_scott_loss(uN, vN, u_target, v_target)


# ------------------------------------------- semi-implicit Fourier spectral solver (Sec. 2.4.2)
#
# The paper's second solver: write dpsi/dt = L psi + sum_i N_i f_i(psi) with L and N_i linear
# operators; in Fourier space (grad -> i k, lap -> -|k|^2) integrate the linear part exactly
# over a step and hold the nonlinear terms fixed:
#   psi_k(t + dt) = A psi_k(t) + B sum_i N_i(k) f_i(psi)_k,  A = exp(L dt),  B = (A - 1) / L
# (B -> dt where L = 0).  Splits used here, all on the periodic grid of spacing h:
#   Model A: L = -k^2 + c1,             N = 1,       f = -c2 psi^3
#   Model B: L = M (-k^4 + c1 k^2),     N = -M k^2,  f = c2 m^3
#   Model C: psi: L = -k^2 + c1, N = 1, f = -c2 psi^3 + 2 c5 psi m;
#            m:   L = -k^4 + c3 k^2, N = -k^2, f = c4 m^3 - c5 psi^2

def wavenumber_sq(shape, h: float = 1.0):
    """|k|^2 on the real-to-complex FFT grid of ``shape`` (last axis halved)."""
    ks = [2.0 * np.pi * np.fft.fftfreq(n, d=h) for n in shape[:-1]]
    ks.append(2.0 * np.pi * np.fft.rfftfreq(shape[-1], d=h))
    grids = np.meshgrid(*ks, indexing="ij")
    return sum(g * g for g in grids)


def _phi_b(Ldt, dt):
    """(A, B) = (exp(L dt), (exp(L dt) - 1) / L) with the L -> 0 limit B = dt."""
    A = np.exp(Ldt)
    small = np.abs(Ldt) < 1e-12
    B = np.where(small, dt * (1.0 + 0.5 * Ldt), np.expm1(Ldt) / np.where(small, 1.0, Ldt / dt))
    return A, B


def spectral_operators(model: str, shape, coeffs, dt: float, h: float = 1.0):
    """Per field (A(k), B(k) N(k)) arrays of the semi-implicit scheme."""
    k2 = wavenumber_sq(shape, h)
    if model == "ac":
        c1, c2 = coeffs
        A, B = _phi_b((-k2 + c1) * dt, dt)
        return [(A, B)]
    if model == "ch":
        c1, c2, M = coeffs
        A, B = _phi_b(M * (-k2 * k2 + c1 * k2) * dt, dt)
        return [(A, B * (-M * k2))]
    if model == "c":
        c1, c2, c3, c4, c5 = coeffs
        Ap, Bp = _phi_b((-k2 + c1) * dt, dt)
        Am, Bm = _phi_b((-k2 * k2 + c3 * k2) * dt, dt)
        return [(Ap, Bp), (Am, Bm * (-k2))]
    raise ValueError(f"the spectral solver takes models ac, ch, c (got {model!r})")


def spectral_nonlinear(model: str, fields, coeffs):
    """The nonlinear terms f_i (real space), one per field."""
    if model == "ac":
        c1, c2 = coeffs
        return [-c2 * fields[0] ** 3]
    if model == "ch":
        c1, c2, M = coeffs
        return [c2 * fields[0] ** 3]
    c1, c2, c3, c4, c5 = coeffs
    psi, m = fields
    return [-c2 * psi ** 3 + 2.0 * c5 * psi * m, c4 * m ** 3 - c5 * psi ** 2]


def spectral_run(model: str, fields, coeffs, dt: float, n_steps: int, h: float = 1.0):
    """``n_steps`` semi-implicit spectral steps (Sec. 2.4.2) in FP64."""
    x = tuple(_f64(f) for f in fields)
    shape = x[0].shape
    ops = spectral_operators(model, shape, coeffs, dt, h)
    axes = tuple(range(len(shape)))
    for _ in range(int(n_steps)):
        nl = spectral_nonlinear(model, x, coeffs)
        new = []
        for xi, fi, (A, BN) in zip(x, nl, ops):
            xk = np.fft.rfftn(xi, axes=axes)
            fk = np.fft.rfftn(fi, axes=axes)
            new.append(np.fft.irfftn(A * xk + BN * fk, s=shape, axes=axes))
        x = tuple(new)
    return x


def structure_factor(psi, h: float = 1.0, n_bins: int = 32):
    """Radially averaged S(k) = |rho_k|^2 / N of rho = 1 where psi > 0, else 0 (Sec. 3).

    Uses the full (not half) spectrum; bins of width k_max / n_bins over |k| in
    (0, k_max], k_max = pi / h * sqrt(d).  Returns (bin centres, mean S per bin, counts).
    """
    psi = _f64(psi)
    rho = (psi > 0).astype(np.float64)
    rk = np.fft.fftn(rho)
    S = (rk * np.conj(rk)).real / rho.size
    ks = np.meshgrid(*[2.0 * np.pi * np.fft.fftfreq(n, d=h) for n in psi.shape], indexing="ij")
    kmag = np.sqrt(sum(k * k for k in ks))
    kmax = np.pi / h * np.sqrt(psi.ndim)
    idx = np.floor(kmag / kmax * n_bins).astype(np.int64)
    idx = np.minimum(idx, n_bins - 1)
    valid = kmag > 0
    sums = np.bincount(idx[valid], weights=S[valid], minlength=n_bins)
    counts = np.bincount(idx[valid], minlength=n_bins)
    centres = (np.arange(n_bins) + 0.5) * kmax / n_bins
    with np.errstate(invalid="ignore", divide="ignore"):
        mean = np.where(counts > 0, sums / np.maximum(counts, 1), 0.0)
    return centres, mean, counts


def porod_fit(centres, mean, counts, k_lo: float, k_hi: float):
    """Least-squares line log S = slope log k + intercept through the bins with centres in
    [k_lo, k_hi], a non-zero count and S > 0: the Porod-law check of Sec. 3 (Eq. for Porod's
    law, S ~ k^-(d+1)). Returns (slope, intercept, bins used)."""
    xs, ys = [], []
    for c, m, n in zip(centres, mean, counts):
        if k_lo <= c <= k_hi and n > 0 and m > 0:
            xs.append(np.log(float(c)))
            ys.append(np.log(float(m)))
    n = len(xs)
    if n < 2:
        raise ValueError("fewer than two usable bins in the window")
    xbar = sum(xs) / n
    ybar = sum(ys) / n
    sxy = sum((x - xbar) * (y - ybar) for x, y in zip(xs, ys))
    sxx = sum((x - xbar) * (x - xbar) for x in xs)
    slope = sxy / sxx
    return slope, ybar - slope * xbar, n
