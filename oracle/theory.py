"""Closed forms and exact moment recursions for the discrete scheme.

TEST INFRASTRUCTURE ONLY.  These formulas pin the C oracle to mathematics
that is independent of its code path: they never draw a random number and
never step a sample path.

* Deterministic limit (alpha = 0, Sec. 3): the forward-Euler step with the
  Dirichlet wall stencil of Eq. (3.8) is diagonalised exactly by the
  half-shifted sine modes sin(m pi (i+1/2)/N) (the wall stencil is the
  centred stencil with an antisymmetric ghost cell), eigenvalue
  1 - 4 r sin^2(m pi / 2N); periodic grids by Fourier modes, eigenvalue
  1 - 4 r sin^2(pi k / N).
* Exact first and second moments of the stochastic step.  The face noise is
  independent of the state at the start of the step (the Ito reading of the
  scheme, Sec. 3), so with T' = A T + b + sum_f g_f(T) N_f d_f:
      m' = A m + b
      C' = A C A^T + sum_f E[g_f^2] d_f d_f^T
  with E[g_f^2] = 2 r eps w_f^2 ((P_f m + q_f)^2 + P_f C P_f^T) for heat
  (noise proportional to the face temperature, Eq. (2.12)) and
  2 r eps w_f^2 (P_f m + q_f) for species (noise proportional to the square
  root of the face concentration, Eq. (4.7)).  This closure is exact.
* Stationary covariance of that recursion (discrete Lyapunov equation,
  the discrete-time analogue of the fluctuation-dissipation relation of
  the supplement, Eq. (SM1.6)).
* Predictor-corrector scheme (Sec. 3: the forward-Euler step as predictor
  T*, then T' = (T + T* + D(T*) + div G(T*)) / 2 with the same face noise).
  With F_N = A + sum_f s_f N_f d_f P_f^T and g_N = b + sum_f s_f N_f q_f d_f
  the heat step is T* = F_N T + g_N and T' = (I + F_N^2) T / 2 +
  (I + F_N) g_N / 2: affine in T with coefficients polynomial (degree <= 2)
  in the step's normals, which are independent of T.  The first two moments
  therefore propagate exactly, and tensor Gauss-Hermite quadrature with 3
  nodes per face (exact to degree 5 per variable) evaluates the expectations
  exactly; applied to forward Euler it reproduces the closed recursion above.
  Deterministic modes are amplified by 1 - x + x^2/2 (Heun) instead of 1 - x,
  x = r mu; with additive noise the stationary structure factor is
  eps T^2 N (2 - x) / (2 - x + x^2/2), an O(x^2) deviation from the flat
  value where forward Euler's is O(x) (the error orders the paper states in
  its exercises, Sec. 6).
* Closed forms: forward-Euler equilibrium covariance
  eps T^2 (I + r L / 2)^{-1}, whose r -> 0 limit is eps T^2 I (Eq. (3.10));
  periodic structure factor eps T^2 N / (1 - r mu_k / 2) whose r -> 0 limit is
  the flat S_k = eps T^2 N (Eq. (3.12), with the cell volume restored);
  the non-equilibrium long-range correlation of Eq. (3.13).
"""
import numpy as np
import scipy.linalg


# --------------------------------------------------------------- operators --

def laplacian_1d(N, bc):
    """Matrix L of the second-difference stencil (without the r factor):
    interior T_{i+1} - 2 T_i + T_{i-1}; Dirichlet end cells -3 on the
    diagonal (Eq. (3.8), wall values enter through the vector b);
    periodic wrap."""
    L = np.zeros((N, N))
    for i in range(N):
        L[i, i] = -2.0
        if i > 0:
            L[i, i - 1] += 1.0
        elif bc == "periodic":
            L[i, N - 1] += 1.0
        if i < N - 1:
            L[i, i + 1] += 1.0
        elif bc == "periodic":
            L[i, 0] += 1.0
    if bc == "dirichlet":
        L[0, 0] = -3.0
        L[N - 1, N - 1] = -3.0
    return L


def faces_1d(N, bc, wall_lo, wall_hi):
    """List of faces (P_f, q_f, w2_f, d_f): face value P_f.T + q_f, squared
    wall weight w_f^2 (2 at Dirichlet walls, Sec. 3), and divergence vector
    d_f (flux through face f leaves cell f and enters cell f-1, Eq. (3.3))."""
    out = []
    nf = N + 1 if bc == "dirichlet" else N
    for f in range(nf):
        P = np.zeros(N)
        d = np.zeros(N)
        q = 0.0
        w2 = 1.0
        if bc == "dirichlet" and f == 0:
            q, w2 = wall_lo, 2.0
        elif bc == "dirichlet" and f == N:
            q, w2 = wall_hi, 2.0
        else:
            P[(f - 1) % N] += 0.5
            P[f % N] += 0.5
        if f < N:
            d[f] -= 1.0
        if f > 0:
            d[f - 1] += 1.0
        elif bc == "periodic":
            d[N - 1] += 1.0
        out.append((P, q, w2, d))
    return out


def laplacian_nd_periodic(shape):
    """Periodic second-difference matrix summed over axes; cell index
    x0 + n0*(x1 + n1*x2) with axis 0 fastest."""
    n = int(np.prod(shape))
    L = np.zeros((n, n))
    dims = list(shape)
    for i in range(n):
        x = np.unravel_index(i, tuple(reversed(dims)))[::-1]
        for a in range(len(dims)):
            for s in (-1, 1):
                y = list(x)
                y[a] = (y[a] + s) % dims[a]
                j = int(np.ravel_multi_index(tuple(reversed(y)), tuple(reversed(dims))))
                L[i, j] += 1.0
            L[i, i] -= 2.0
    return L


def faces_nd_periodic(shape):
    n = int(np.prod(shape))
    dims = list(shape)
    out = []
    for a in range(len(dims)):
        for i in range(n):
            x = np.unravel_index(i, tuple(reversed(dims)))[::-1]
            y = list(x)
            y[a] = (y[a] - 1) % dims[a]
            j = int(np.ravel_multi_index(tuple(reversed(y)), tuple(reversed(dims))))
            P = np.zeros(n)
            P[i] += 0.5
            P[j] += 0.5
            d = np.zeros(n)
            d[i] -= 1.0
            d[j] += 1.0
            out.append((P, 0.0, 1.0, d))
    return out


def face_conductance(cond, bc):
    """Face conductance numbers of a rod of several materials, a[f] for the
    low face of cell f (f = 0..N): the harmonic mean of the two cells' (two
    half-cell resistances in series), the edge cell's own at a Dirichlet wall,
    and face N = face 0 on a periodic rod."""
    c = np.asarray(cond, dtype=float)
    N = len(c)
    a = np.empty(N + 1)
    a[1:N] = 2.0 * c[:-1] * c[1:] / (c[:-1] + c[1:])
    if bc == "dirichlet":
        a[0], a[N] = c[0], c[-1]
    else:
        a[0] = a[N] = 2.0 * c[-1] * c[0] / (c[-1] + c[0])
    return a


def conductance_matrix(a, bc):
    """Matrix L of the conducted heat, (L T)_i = sum over the faces of cell i
    of a_f (T_neighbour - T_i); a Dirichlet wall face conducts over half a
    cell, 2 a_w (T_wall - T_edge), whose T_edge part is on the diagonal."""
    N = len(a) - 1
    L = np.zeros((N, N))
    for f in range(N + 1 if bc == "dirichlet" else N):
        if bc == "dirichlet" and f in (0, N):
            i = 0 if f == 0 else N - 1
            L[i, i] -= 2.0 * a[f]
            continue
        lo, hi = (f - 1) % N, f % N
        L[lo, lo] -= a[f]
        L[hi, hi] -= a[f]
        L[lo, hi] += a[f]
        L[hi, lo] += a[f]
    return L


def _scheme_var(prob_like):
    """(A, b, faces, tref, L) of a rod of several materials (the iron /
    aluminium exercise, Sec. 6): T' = T + C^{-1} (L T + b_w + sum_f g_f N_f
    D_f) with C = diag(rho c_V,i), L the conductance matrix, b_w the walls'
    conducted heat and E[g_f^2] = 2 k_B a_f / dV x E[T_f^2] (x 2 at a wall:
    its half-cell conductance is 2 a_w).  Faces carry that full coefficient
    in place of the squared wall weight."""
    N = prob_like["n"][0]
    bc = prob_like["bc"]
    cond = np.asarray(prob_like["cond"], dtype=float)
    cap = np.asarray(prob_like["cap"], dtype=float)
    kb_dv = prob_like["kB_dV"]
    a = face_conductance(cond, bc)
    L = conductance_matrix(a, bc)
    bw = np.zeros(N)
    if bc == "dirichlet":
        bw[0] = 2.0 * a[0] * prob_like["wall_lo"]
        bw[-1] = 2.0 * a[N] * prob_like["wall_hi"]
    A = np.eye(N) + L / cap[:, None]
    b = bw / cap
    faces = []
    for P, q, w2, d in faces_1d(N, bc, prob_like["wall_lo"], prob_like["wall_hi"]):
        f = len(faces)
        faces.append((P, q, 2.0 * kb_dv * a[f] * w2, d / cap))
    if bc == "dirichlet":
        tref = np.linalg.solve(np.eye(N) - A, b)
    else:
        tref = np.full(N, float(prob_like["wall_lo"]))
    return A, b, faces, tref, L


def variable_equilibrium_cov(cond, cap, kb_dv, bc, T):
    """Forward-Euler equilibrium covariance of a rod of several materials at
    uniform temperature T with the noise linearised about T:
    k_B T^2 / dV (C - L/2)^{-1}, C = diag(rho c_V,i), L the conductance
    matrix (negative semi-definite).  Derivation: with A = I + C^{-1} L and
    Q = 2 k_B T^2 / dV C^{-1} (-L) C^{-1} (the fluctuation-dissipation
    balance of each face), X = (C + L/2)^{-1} solves
    X = A X A^T + 2 C^{-1} (-L) C^{-1}, because with B = C + L/2,
    (B + L/2) B^{-1} (B + L/2) = (B - L/2) B^{-1} (B - L/2) - 2 L.  Its
    r -> 0 limit is k_B T^2 / (rho c_V,i dV) per cell and no correlation
    (Eq. (3.10) per material).  Periodic rods conserve the energy
    sum rho c_V,i T_i, and X + alpha 1 1^T solves the same equation; since
    1^T (C + L/2) = c^T, c^T X = 1^T, and the solution with no energy
    fluctuation (c^T S = 0) is X - 1 1^T / sum_i rho c_V,i."""
    a = face_conductance(cond, bc)
    L = conductance_matrix(a, bc)
    c = np.asarray(cap, dtype=float)
    X = np.linalg.inv(np.diag(c) + 0.5 * L)
    if bc != "dirichlet":
        n = len(c)
        X = X - np.ones((n, n)) / c.sum()
    return kb_dv * T * T * X


def scheme(prob_like):
    """(A, b, faces, tref) of one forward-Euler step for a problem given as a
    dict with dim, n, bc, r, eps, wall_lo, wall_hi, equation (and, for a rod
    of several materials, cond, cap and kB_dV in place of r and eps)."""
    if prob_like.get("cond") is not None:
        return _scheme_var(prob_like)
    dim = prob_like["dim"]
    r = prob_like["r"]
    if dim == 1:
        N = prob_like["n"][0]
        bc = prob_like["bc"]
        L = laplacian_1d(N, bc)
        b = np.zeros(N)
        if bc == "dirichlet":
            b[0] = 2.0 * r * prob_like["wall_lo"]
            b[-1] = 2.0 * r * prob_like["wall_hi"]
            x = (np.arange(N) + 0.5) / N
            tref = prob_like["wall_lo"] + (prob_like["wall_hi"] - prob_like["wall_lo"]) * x
        else:
            tref = np.full(N, float(prob_like["wall_lo"]))
        faces = faces_1d(N, bc, prob_like["wall_lo"], prob_like["wall_hi"])
    else:
        shape = tuple(prob_like["n"][:dim])
        L = laplacian_nd_periodic(shape)
        b = np.zeros(L.shape[0])
        tref = np.full(L.shape[0], float(prob_like["wall_lo"]))
        faces = faces_nd_periodic(shape)
    A = np.eye(L.shape[0]) + r * L
    theta = {"be": 1.0, "cn": 0.5}.get(prob_like.get("scheme", "fe"))
    if theta is not None:
        # implicit diffusion with weight theta, explicit noise (the implicit
        # exercise of Sec. 6): T' = M^{-1} ((I + (1 - theta) r L) T + b + sum_f g_f d_f),
        # M = I - theta r L; the face values are still those of T
        Minv = np.linalg.inv(np.eye(L.shape[0]) - theta * r * L)
        A = Minv @ (np.eye(L.shape[0]) + (1.0 - theta) * r * L)
        b = Minv @ b
        faces = [(P, q, w2, Minv @ d) for P, q, w2, d in faces]
    return A, b, faces, tref, L


def noise_cov(prob_like, faces, m, C):
    """sum_f E[g_f^2] d_f d_f^T for mean m and covariance C of the state."""
    var = prob_like.get("cond") is not None
    r, eps = (1.0, 0.5) if var else (prob_like["r"], prob_like["eps"])   # var: the face holds 2 r eps w2
    heat = prob_like.get("equation", "heat") == "heat"
    n = len(m)
    Q = np.zeros((n, n))
    for P, q, w2, d in faces:
        fm = P @ m + q
        if heat:
            e = 2.0 * r * eps * w2 * (fm * fm + P @ C @ P)
        else:
            e = 2.0 * r * eps * w2 * fm
        Q += e * np.outer(d, d)
    return Q


def initial_moments(prob_like, tref):
    """Mean and covariance of the seeded initial condition: T_ref plus iid
    sigma*N(0,1) (sigma^2 = eps*T_mid^2 heat, eps*c_mid species), projected
    to zero sum on periodic grids."""
    n = len(tref)
    C = np.zeros((n, n))
    if prob_like.get("perturb_ic", 1) and prob_like.get("cond") is not None:
        # each cell's own equilibrium variance k_B T_mid^2 / (rho c_V,i dV);
        # periodic: projected to zero energy sum rho c_V,i delta_i
        mid = 0.5 * (prob_like["wall_lo"] + prob_like["wall_hi"])
        cap = np.asarray(prob_like["cap"], dtype=float)
        C = np.diag(prob_like["kB_dV"] * mid * mid / cap)
        if prob_like["bc"] == "periodic":
            Pr = np.eye(n) - np.outer(np.ones(n), cap) / cap.sum()
            C = Pr @ C @ Pr.T
        return tref.copy(), C
    if prob_like.get("perturb_ic", 1):
        mid = 0.5 * (prob_like["wall_lo"] + prob_like["wall_hi"])
        if prob_like.get("equation", "heat") == "heat":
            s2 = prob_like["eps"] * mid * mid
        else:
            s2 = prob_like["eps"] * abs(mid)
        C = s2 * np.eye(n)
        if prob_like["dim"] > 1 or prob_like["bc"] == "periodic":
            Pr = np.eye(n) - np.ones((n, n)) / n
            C = Pr @ C @ Pr
    return tref.copy(), C


def pooled_expectation(prob_like, nsteps, K, relax, step0=0):
    """Exact expectation of the pooled sample statistics the oracle and the
    GPU accumulate over steps step0+1..step0+nsteps (sample at step m iff
    m % K == 0 and m > relax): returns dict with E[mean delta], E[second
    moment of delta] (matrix), per-sample list not kept."""
    A, b, faces, tref, _ = scheme(prob_like)
    m, C = initial_moments(prob_like, tref)
    n = len(m)
    s1 = np.zeros(n)
    s2 = np.zeros((n, n))
    cnt = 0
    for mstep in range(step0 + 1, step0 + nsteps + 1):
        Q = noise_cov(prob_like, faces, m, C)
        C = A @ C @ A.T + Q
        m = A @ m + b
        if mstep % K == 0 and mstep > relax:
            dm = m - tref
            s1 += dm
            s2 += C + np.outer(dm, dm)
            cnt += 1
    return {"count": cnt, "mean_delta": s1 / cnt, "second": s2 / cnt,
            "final_mean": m, "final_cov": C, "tref": tref}


def stationary(prob_like, iters=50):
    """Stationary mean and covariance of the exact moment recursion: the
    mean solves m = A m + b; the covariance solves the discrete Lyapunov
    equation C = A C A^T + Q(m, C), iterated on the (small, O(eps))
    multiplicative part of Q."""
    A, b, faces, tref, L = scheme(prob_like)
    n = len(tref)
    periodic = prob_like["dim"] > 1 or prob_like["bc"] == "periodic"
    if periodic and prob_like.get("cond") is not None:
        m = tref.copy()
        cap = np.asarray(prob_like["cap"], dtype=float)
        Pr = np.eye(n) - np.outer(np.ones(n), cap) / cap.sum()
    elif periodic:
        m = tref.copy()
        Pr = np.eye(n) - np.ones((n, n)) / n
    else:
        m = np.linalg.solve(np.eye(n) - A, b)
        Pr = np.eye(n)
    C = np.zeros((n, n))
    # project the zero mode out (the total is conserved on periodic grids)
    Ap = Pr @ A @ Pr
    for _ in range(iters):
        Q = Pr @ noise_cov(prob_like, faces, m, C) @ Pr.T
        Cn = scipy.linalg.solve_discrete_lyapunov(Ap, Q)
        Cn = 0.5 * (Cn + Cn.T)
        if np.max(np.abs(Cn - C)) <= 1e-15 * max(1.0, np.max(np.abs(Cn))):
            C = Cn
            break
        C = Cn
    return m, C


# ---------------------------------------------------------- closed forms --

def fe_equilibrium_cov(N, bc, r, eps, T):
    """Linearised forward-Euler equilibrium covariance eps T^2 (I + r L/2)^{-1}
    (Dirichlet), which tends to eps T^2 I (Eq. (3.10)) as r -> 0; on
    periodic grids the zero mode is removed."""
    L = laplacian_1d(N, bc)
    M = np.eye(N) + 0.5 * r * L
    if bc == "dirichlet":
        return eps * T * T * np.linalg.inv(M)
    Pr = np.eye(N) - np.ones((N, N)) / N
    return eps * T * T * Pr @ np.linalg.pinv(Pr @ M @ Pr) @ Pr


def fe_structure_factor(shape, r, eps_amp):
    """Periodic forward-Euler structure factor for k != 0:
    eps_amp * Ncells / (1 - r mu_k / 2), mu_k = sum_axes 4 sin^2(pi k_a/n_a).
    eps_amp = eps T^2 (heat, linearised) or eps c (species, exact).
    Array ordered like the cells (axis 0 fastest); entry k = 0 is set to 0."""
    dims = list(shape)
    ncell = int(np.prod(dims))
    grids = np.meshgrid(*[np.arange(n) for n in reversed(dims)], indexing="ij")
    mu = np.zeros(grids[0].shape)
    for g, n in zip(grids, reversed(dims)):
        mu += 4.0 * np.sin(np.pi * g / n) ** 2
    S = eps_amp * ncell / (1.0 - 0.5 * r * mu)
    S = S.ravel()
    S[0] = 0.0
    return S


def fe_structure_factor_transient(shape, r, eps_amp, nsteps):
    """S_k after n steps from a uniform state: S_inf (1 - lambda_k^{2n}),
    lambda_k = 1 - r mu_k."""
    dims = list(shape)
    grids = np.meshgrid(*[np.arange(n) for n in reversed(dims)], indexing="ij")
    mu = np.zeros(grids[0].shape)
    for g, n in zip(grids, reversed(dims)):
        mu += 4.0 * np.sin(np.pi * g / n) ** 2
    lam = (1.0 - r * mu).ravel()
    S = fe_structure_factor(shape, r, eps_amp)
    return S * (1.0 - lam ** (2 * nsteps))


def periodic_variance(N, r, eps_amp):
    """Pointwise variance on a periodic 1D FE grid: (1/N^2) sum_{k!=0} S_k;
    tends to eps_amp (1 - 1/N) (the conservation correction of Sec. 3) as r -> 0."""
    S = fe_structure_factor((N,), r, eps_amp)
    return S.sum() / (N * N)


def long_range_correlation(N, eps, dT):
    """Non-equilibrium long-range part of Eq. (3.13) in cell units:
    eps (dT)^2 (i+1/2)(N-j-1/2)/N^3 for i <= j (symmetric)."""
    x = np.arange(N) + 0.5
    lo = np.minimum.outer(x, x)
    hi = np.maximum.outer(x, x)
    return eps * dT * dT * lo * (N - hi) / N ** 3


def amplification(x, scheme="fe"):
    """Deterministic factor per step of a mode with eigenvalue -x of r L:
    forward Euler 1 - x; predictor-corrector (Heun) 1 - x + x^2/2; the
    implicit theta scheme (1 - (1 - theta) x) / (1 + theta x), theta = 1
    backward Euler, 1/2 Crank-Nicolson (|factor| <= 1 for every x >= 0: both
    unconditionally stable)."""
    x = np.asarray(x, dtype=float)
    theta = {"be": 1.0, "cn": 0.5}.get(scheme)
    if theta is not None:
        return (1.0 - (1.0 - theta) * x) / (1.0 + theta * x)
    return 1.0 - x + (0.5 * x * x if scheme == "pc" else 0.0)


def sine_mode_solution(N, r, wall_lo, wall_hi, T0, nsteps, scheme="fe"):
    """Exact deterministic forward-Euler solution with Dirichlet walls:
    T^n = T_lin + sum_m b_m lambda_m^n sin(m pi (i+1/2)/N),
    lambda_m = 1 - 4 r sin^2(m pi/(2N)), b from the initial deviation."""
    i = np.arange(N)
    x = (i + 0.5) / N
    tlin = wall_lo + (wall_hi - wall_lo) * x
    m = np.arange(1, N + 1)
    Phi = np.sin(np.pi * np.outer(i + 0.5, m) / N)       # [cell, mode]
    bm = np.linalg.solve(Phi, np.asarray(T0) - tlin)
    lam = amplification(4.0 * r * np.sin(m * np.pi / (2.0 * N)) ** 2, scheme)
    return tlin + Phi @ (bm * lam ** nsteps)


def fourier_mode_solution(N, r, T0, nsteps, scheme="fe"):
    """Exact deterministic solution on a periodic grid: each Fourier mode is
    multiplied per step by the scheme's amplification of
    x = 4 r sin^2(pi k/N)."""
    k = np.arange(N)
    lam = amplification(4.0 * r * np.sin(np.pi * k / N) ** 2, scheme)
    That = np.fft.fft(np.asarray(T0))
    return np.real(np.fft.ifft(That * lam ** nsteps))


def structure_factor(shape, r, eps_amp, scheme="fe"):
    """Periodic structure factor for k != 0 with additive noise (the
    linearised heat equation; exact for species): forward Euler
    eps_amp N / (1 - x/2), predictor-corrector eps_amp N (2 - x) /
    (2 - x + x^2/2), backward Euler eps_amp N / (1 + x/2), Crank-Nicolson
    eps_amp N, x = r mu_k (derivation: per mode T' = g T + h eta with
    g = 1 - x + x^2/2 and h = 1 - x/2, so S = h^2 sigma^2 / (1 - g^2)).
    Entry k = 0 is set to 0; cells ordered with axis 0 fastest."""
    dims = list(shape)
    ncell = int(np.prod(dims))
    grids = np.meshgrid(*[np.arange(n) for n in reversed(dims)], indexing="ij")
    mu = np.zeros(grids[0].shape)
    for g, n in zip(grids, reversed(dims)):
        mu += 4.0 * np.sin(np.pi * g / n) ** 2
    x = r * mu
    if scheme == "pc":
        S = eps_amp * ncell * (2.0 - x) / (2.0 - x + 0.5 * x * x)
    elif scheme in ("be", "cn"):
        # implicit theta scheme: per mode S = q / ((1 + theta x)^2 - (1 - (1 - theta) x)^2)
        # with the forward-Euler noise q = 2 x eps_amp N, i.e.
        # eps_amp N / (1 + (theta - 1/2) x): Crank-Nicolson gives the flat value
        # at every time step, backward Euler falls below it
        theta = 1.0 if scheme == "be" else 0.5
        S = eps_amp * ncell / (1.0 + (theta - 0.5) * x)
    else:
        S = eps_amp * ncell / (1.0 - 0.5 * x)
    S = S.ravel()
    S[0] = 0.0
    return S



# ------------------------------------ structure factors pooled over samples --

def _sample_steps(K, relax, nsteps, step0=0):
    """Sampling steps m (1-based) of a run of steps step0+1..step0+nsteps:
    m % K == 0 and m > relax (Sec. 3, Eq. (3.9), after relaxation)."""
    lo = max(step0, relax) // K + 1
    hi = (step0 + nsteps) // K
    return np.arange(lo, hi + 1, dtype=np.float64) * K


def _mean_power(lam2, ns):
    """Mean over the sample times n of lam2^n (lam2 = lambda^2 in [0, 1]);
    the times are an arithmetic progression n_1 + K j, j < M, so the mean is
    the geometric sum lam2^{n_1} (1 - q^M) / (M (1 - q)), q = lam2^K (1 where
    q = 1), with the ratio taken through expm1 for q near 1."""
    ns = np.asarray(ns, dtype=np.float64)
    M = len(ns)
    if M == 0:
        return np.zeros_like(lam2)
    n1 = ns[0]
    step = ns[1] - ns[0] if M > 1 else 1.0
    assert M == 1 or np.all(np.diff(ns) == step)
    lam2 = np.asarray(lam2, dtype=np.float64)
    with np.errstate(divide="ignore", invalid="ignore", over="ignore"):
        lg = np.log(lam2)                       # -inf where lam2 = 0
        first = np.exp(n1 * lg)
        num = -np.expm1(M * step * lg)
        den = -np.expm1(step * lg)
        ratio = np.where(den > 0.0, num / np.where(den > 0.0, den, 1.0) / M, 1.0)
    return np.where(lam2 > 0.0, first * ratio, 0.0)


def fe_structure_factor_pooled(shape, r, eps_amp, s0, K, relax, nsteps, step0=0):
    """Exact expectation of the structure factor <|hat delta_k|^2> pooled over
    the sampling steps of a run (sample at m iff m % K == 0 and m > relax) on
    a periodic grid stepped by forward Euler with noise of constant expected
    strength -- species, whose face-noise variance 2 r eps_c E[c_f] is linear
    in the state, so that with the conserved uniform mean c the per-mode
    recursion S' = lambda^2 S + q is exact (eps_amp = eps_c c).  From S_k = s0
    at step step0 (the seeded initial perturbation: s0 = sigma^2 x cells for
    k != 0), S_k(n) = S_inf + (s0 - S_inf) lambda_k^{2 (n - step0)},
    lambda_k = 1 - r mu_k, S_inf = eps_amp cells / (1 - r mu_k / 2)
    (fe_structure_factor).  Cells order, axis 0 fastest; k = 0 set to 0."""
    dims = list(shape)
    grids = np.meshgrid(*[np.arange(n) for n in reversed(dims)], indexing="ij")
    mu = np.zeros(grids[0].shape)
    for g, n in zip(grids, reversed(dims)):
        mu += 4.0 * np.sin(np.pi * g / n) ** 2
    lam2 = ((1.0 - r * mu) ** 2).ravel()
    S_inf = fe_structure_factor(shape, r, eps_amp)
    ns = _sample_steps(K, relax, nsteps, step0) - step0
    out = S_inf + (s0 - S_inf) * _mean_power(lam2, ns)
    out[0] = 0.0
    return out


def _axis_mus(dims):
    """Per-axis mu_a(k_a) = 4 sin^2(pi k_a / n_a)."""
    return [4.0 * np.sin(np.pi * np.arange(n) / n) ** 2 for n in dims]


def heat_face_variance(shape, r, eps, T0):
    """Stationary variance v_a of a face value (T_i + T_{i - e_a}) / 2 along
    each axis a on a periodic heat grid at uniform mean T0.  The heat face
    noise has E[g_f^2] = 2 r eps E[T_f^2] = 2 r eps (T0^2 + v_a) (noise
    proportional to the face temperature, Eq. (2.12)), so per Fourier mode
    S_k = 2 r eps cells sum_a (T0^2 + v_a) mu_a(k) / (1 - lambda_k^2), while
    v_a = (1/cells^2) sum_k S_k cos^2(pi k_a / n_a) (the face average's
    transfer function): a linear system for v solved here.  Returns v (one
    entry per axis)."""
    dims = list(shape)
    D = len(dims)
    cells = float(np.prod(dims))
    mus = _axis_mus(dims)
    grids = np.meshgrid(*[np.arange(n) for n in dims], indexing="ij")
    mu_a = [mus[a][grids[a]] for a in range(D)]
    mu = sum(mu_a)
    den = 1.0 - (1.0 - r * mu) ** 2
    den[(0,) * D] = 1.0
    M = np.zeros((D, D))
    for a in range(D):
        cos2 = 1.0 - mu_a[a] / 4.0
        for b in range(D):
            w = cos2 * mu_a[b] / den
            w[(0,) * D] = 0.0
            M[a, b] = 2.0 * r * eps / cells * w.sum()
    return np.linalg.solve(np.eye(D) - M, M @ np.full(D, T0 * T0))


def heat_axes_structure_factor_pooled(shape, r, eps, T0, K, relax, nsteps, step0=0):
    """Expected per-axis structure factor of a periodic heat grid started
    uniform at T0 (no perturbation), pooled over the sampling steps of a run
    (sample at m iff m % K == 0 and m > relax): for each axis a the 1D DFT
    along a, <|hat delta_line(k_a)|^2> averaged over all lines along a.  By
    Parseval over the other axes this is (1/lines^2) sum over the other
    wavenumbers of the full-grid <|hat delta_k|^2>, which from a uniform start
    is S_inf,k (1 - lambda_k^{2 n}) with the face noise strength
    2 r eps (T0^2 + v_b) on axis b (multiplicative noise, Eq. (2.12)):
    S_inf,k = 2 r eps cells sum_b (T0^2 + v_b) mu_b(k) / (1 - lambda_k^2).
    The face variance is taken at its stationary value v_b
    (heat_face_variance) from the first step on: it relaxes within the
    decay time of the high-wavenumber modes that carry it (tens of steps), so
    the neglected part is of order v x (those steps) / (sampled steps)
    relative.  Returns the axes back to back (n_0 + n_1 + ...)."""
    dims = list(shape)
    D = len(dims)
    cells = float(np.prod(dims))
    v = heat_face_variance(shape, r, eps, T0)
    mus = _axis_mus(dims)
    ns = _sample_steps(K, relax, nsteps, step0) - step0
    out = []
    for a in range(D):
        lines = cells / dims[a]
        acc = np.zeros(dims[a])
        # sum over the other axes' wavenumbers, chunked over the outermost
        other = [b for b in range(D) if b != a]
        grids = np.meshgrid(*[mus[b] for b in other], indexing="ij") if other else []
        mu_o = sum(grids) if other else np.zeros(())
        noise_o = sum((T0 * T0 + v[b]) * grids[i] for i, b in enumerate(other)) if other else np.zeros(())
        for ka in range(dims[a]):
            mu = mus[a][ka] + mu_o
            lam2 = (1.0 - r * mu) ** 2
            num = 2.0 * r * eps * cells * ((T0 * T0 + v[a]) * mus[a][ka] + noise_o)
            den = 1.0 - lam2
            with np.errstate(divide="ignore", invalid="ignore"):
                S_inf = np.where(mu > 0.0, num / np.where(mu > 0.0, den, 1.0), 0.0)
            pooled = S_inf * (1.0 - _mean_power(lam2, ns))
            acc[ka] = pooled.sum() / (lines * lines)
        out.append(acc)
    return np.concatenate(out)


# ------------------------------------------- exact moments by quadrature --

def gauss_hermite(nvars, npts):
    """Tensor Gauss-Hermite rule for nvars independent N(0,1) variables:
    (weights [Q], nodes [Q, nvars]); exact for polynomials of degree
    <= 2 npts - 1 in each variable."""
    x, w = np.polynomial.hermite_e.hermegauss(npts)
    w = w / np.sqrt(2.0 * np.pi)
    grids = np.meshgrid(*([np.arange(npts)] * nvars), indexing="ij")
    idx = np.stack([g.ravel() for g in grids], axis=1)
    return np.prod(w[idx], axis=1), x[idx]


def _increment(prob_like, Aminus, b, faces, T, z):
    """D(T) + div G(T) for face normals z (wall weights applied here)."""
    r, eps = prob_like["r"], prob_like["eps"]
    heat = prob_like.get("equation", "heat") == "heat"
    out = Aminus @ T + b
    for (P, q, w2, d), zf in zip(faces, z):
        fv = P @ T + q
        amp = np.sqrt(2.0 * r * eps * w2) * fv if heat else np.sqrt(2.0 * r * eps * w2 * max(fv, 0.0))
        out = out + amp * zf * d
    return out


def step_map(prob_like, T, z, ops=None):
    """One step from state T with face normals z: forward Euler, or the
    predictor-corrector scheme when prob_like["scheme"] == "pc"."""
    A, b, faces, _, _ = ops if ops is not None else scheme(prob_like)
    Am = A - np.eye(len(b))
    Ts = T + _increment(prob_like, Am, b, faces, T, z)
    if prob_like.get("scheme", "fe") != "pc":
        return Ts
    return 0.5 * (T + Ts + _increment(prob_like, Am, b, faces, Ts, z))


def affine_step(prob_like, z, ops=None):
    """Heat only: (F, g) with step(T) = F T + g for face normals z."""
    A, b, faces, _, _ = ops if ops is not None else scheme(prob_like)
    r, eps = prob_like["r"], prob_like["eps"]
    F = A.copy()
    g = b.copy()
    for (P, q, w2, d), zf in zip(faces, z):
        s = np.sqrt(2.0 * r * eps * w2) * zf
        F += s * np.outer(d, P)
        g += s * q * d
    if prob_like.get("scheme", "fe") == "pc":
        I = np.eye(len(b))
        return 0.5 * (I + F @ F), 0.5 * (I + F) @ g
    return F, g


def pooled_expectation_quadrature(prob_like, nsteps, K, relax, step0=0):
    """Exact expectation of the pooled statistics (as pooled_expectation) for
    the heat equation under either scheme, propagating E[T] and E[T T^T]
    through the affine random step with 3-node Gauss-Hermite quadrature over
    the faces (exact: the integrands have degree <= 4 per normal)."""
    assert prob_like.get("equation", "heat") == "heat"
    ops = scheme(prob_like)
    tref = ops[3]
    nf = len(ops[2])
    W, Z = gauss_hermite(nf, 3)
    maps = [affine_step(prob_like, z, ops) for z in Z]
    F = np.stack([fg[0] for fg in maps])          # [Q, n, n]
    G = np.stack([fg[1] for fg in maps])          # [Q, n]
    EF = np.einsum("q,qij->ij", W, F)
    Eg = W @ G
    m, C = initial_moments(prob_like, tref)
    S = C + np.outer(m, m)
    n = len(m)
    s1 = np.zeros(n)
    s2 = np.zeros((n, n))
    cnt = 0
    for mstep in range(step0 + 1, step0 + nsteps + 1):
        Fm = F @ m                                 # [Q, n]
        cross = np.einsum("q,qi,qj->ij", W, Fm, G)
        Sn = (np.einsum("q,qij,jk,qlk->il", W, F, S, F, optimize=True) + cross + cross.T
              + np.einsum("q,qi,qj->ij", W, G, G))
        m = EF @ m + Eg
        S = 0.5 * (Sn + Sn.T)
        if mstep % K == 0 and mstep > relax:
            s1 += m - tref
            s2 += S - np.outer(m, tref) - np.outer(tref, m) + np.outer(tref, tref)
            cnt += 1
    C = S - np.outer(m, m)
    return {"count": cnt, "mean_delta": s1 / cnt, "second": s2 / cnt,
            "final_mean": m, "final_cov": C, "tref": tref}


def first_step_quadrature(prob_like, T0, npts):
    """Mean and covariance of one step from the fixed state T0 by npts-node
    Gauss-Hermite quadrature over the faces (exact for heat with npts >= 2;
    for species the integrand is smooth where the face values stay positive,
    and the rule converges rapidly in npts)."""
    ops = scheme(prob_like)
    W, Z = gauss_hermite(len(ops[2]), npts)
    T0 = np.asarray(T0, dtype=float)
    vals = np.array([step_map(prob_like, T0, z, ops) for z in Z])
    mean = W @ vals
    dev = vals - mean
    return mean, (dev * W[:, None]).T @ dev


# ------------------------------------------------------- time correlation --

def mean_map(prob_like, ops=None):
    """(M, g0) with E[T' | T] = M T + g0 for one step: forward Euler A, b
    (the face noise has mean zero and is independent of T); the heat
    predictor-corrector step E[F], E[g] (exact by quadrature).  The
    predictor-corrector species step has no affine conditional mean (the
    corrector's noise amplitude depends on the predictor's noise)."""
    ops = ops if ops is not None else scheme(prob_like)
    A, b, faces = ops[0], ops[1], ops[2]
    if prob_like.get("scheme", "fe") != "pc":
        return A, b
    assert prob_like.get("equation", "heat") == "heat"
    W, Z = gauss_hermite(len(faces), 3)
    maps = [affine_step(prob_like, z, ops) for z in Z]
    return (np.einsum("q,qij->ij", W, np.stack([f for f, g in maps])),
            W @ np.stack([g for f, g in maps]))


def moment_path(prob_like, nsteps, step0=0):
    """E[T] and E[T T^T] after each of nsteps steps (entry 0: the initial
    state): the closed forward-Euler recursion, or for the heat
    predictor-corrector scheme the quadrature recursion."""
    ops = scheme(prob_like)
    A, b, faces, tref, _ = ops
    m, C = initial_moments(prob_like, tref)
    path = [(m.copy(), C + np.outer(m, m))]
    if prob_like.get("scheme", "fe") != "pc":
        for _ in range(nsteps):
            Q = noise_cov(prob_like, faces, m, C)
            C = A @ C @ A.T + Q
            m = A @ m + b
            path.append((m.copy(), C + np.outer(m, m)))
        return path
    assert prob_like.get("equation", "heat") == "heat"
    W, Z = gauss_hermite(len(faces), 3)
    maps = [affine_step(prob_like, z, ops) for z in Z]
    F = np.stack([f for f, g in maps])
    G = np.stack([g for f, g in maps])
    EF, Eg = np.einsum("q,qij->ij", W, F), W @ G
    S = path[0][1]
    for _ in range(nsteps):
        Fm = F @ m
        cross = np.einsum("q,qi,qj->ij", W, Fm, G)
        Sn = (np.einsum("q,qij,jk,qlk->il", W, F, S, F, optimize=True) + cross + cross.T
              + np.einsum("q,qi,qj->ij", W, G, G))
        m = EF @ m + Eg
        S = 0.5 * (Sn + Sn.T)
        path.append((m.copy(), S.copy()))
    return path


def lagged_expectation(prob_like, nsteps, K, relax, L, step0=0):
    """Exact expectation of the pooled time correlation
    <delta_i(t + l K) delta_i(t)> (delta = T - T_ref) over the pairs of
    sampling steps l K apart within one run of steps step0+1..step0+nsteps
    (sample at step m iff m % K == 0 and m > relax), l = 0..L-1.  Because
    E[T^{t+j} | T^t] = M^j T^t + c_j with c_j = sum_{i<j} M^i g0 (mean_map),
    E[T^{t+j} (T^t)^T] = M^j E[T^t (T^t)^T] + c_j E[T^t]^T, whatever the
    noise.  Returns (expectation [L, cells], pairs per realization [L])."""
    ops = scheme(prob_like)
    tref = ops[3]
    n = len(tref)
    M, g0 = mean_map(prob_like, ops)
    path = moment_path(prob_like, nsteps, step0)
    samples = [m for m in range(step0 + 1, step0 + nsteps + 1) if m % K == 0 and m > relax]
    Mj, cj = [np.eye(n)], [np.zeros(n)]
    for _ in range((L - 1) * K):
        cj.append(M @ cj[-1] + g0)
        Mj.append(M @ Mj[-1])
    out = np.zeros((L, n))
    cnt = np.zeros(L)
    for s, ts in enumerate(samples):
        m_s = path[ts - step0][0]
        for l in range(min(L, s + 1)):
            tp = samples[s - l]
            j = ts - tp
            m_p, S_p = path[tp - step0]
            cross = Mj[j] @ S_p + np.outer(cj[j], m_p)
            out[l] += np.diag(cross) - tref * m_p - m_s * tref + tref * tref
            cnt[l] += 1
    return out / np.maximum(cnt, 1)[:, None], cnt
