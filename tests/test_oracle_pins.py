"""Pins of the CPU oracle to things other than itself (CPU only).

Each check is chosen so that a plausible slip in the oracle (a dropped term,
a wrong sign, a transposed gradient, a missing density factor, a wrong
element size h) fails at least one of them:
  * closed forms of single tetrahedra, evaluated with 50-digit decimals;
  * per-term invariants that follow from sum_a grad N_a = 0 and from linearity;
  * textbook special cases: the consistent P1 mass matrix for the Galerkin
    convection, barycentric gradients from an independent linear solve;
  * global identities: divergence theorem on the cube, discrete
    divergence of a constant pressure, rotation/translation/renumbering
    invariance;
  * derivatives: complex step against central differences, the element
    Jacobian VJP against the full complex-step Jacobian and the dot-product
    identity.
"""
import decimal
from decimal import Decimal as D

import numpy as np
import pytest

import meshgen as mg
import oracle

decimal.getcontext().prec = 50
SQ5 = D(5).sqrt()
QA = (D(5) + 3 * SQ5) / 20
QB = (D(5) - SQ5) / 20
REF_DN = [(-1, -1, -1), (1, 0, 0), (0, 1, 0), (0, 0, 1)]


def ref_tet(s=1.0):
    return np.array([[0, 0, 0], [s, 0, 0], [0, s, 0], [0, 0, s]], float)


def closed_form_shear(rho, mu, s, q, c1=4, c2=2):
    """Tet X0=0, Xk=s e_k; u = (y, 1, 0), p = q x, no eddy viscosity.
    grad u has the single entry du/dy = 1, so (u.grad)u = (1, 0, 0) and the
    strong residual is (rho + q, 0, 0); h = s, V = s^3/6, grad N_a = e/s,
    u at Gauss point g: (y_g, 1, 0) with y_g = s*A if g == 2 else s*B,
    p_bar = q s / 4."""
    rho, mu, s, q = D(rho), D(mu), D(s), D(q)
    V = s ** 3 / 6
    h = s
    pbar = q * s / 4
    taus, ys = [], []
    for g in range(4):
        y = s * (QA if g == 2 else QB)
        ys.append(y)
        taus.append(1 / (c1 * mu / h ** 2 + c2 * rho * (y * y + 1).sqrt() / h))
    F = [[D(0)] * 4 for _ in range(4)]
    for a in range(4):
        dN = [D(c) / s for c in REF_DN[a]]
        supg = sum(taus[g] * rho * (ys[g] * dN[0] + dN[1]) * (rho + q) for g in range(4))
        F[a][0] = -V * rho / 4 - V * mu * dN[1] + V * pbar * dN[0] - V / 4 * supg
        F[a][1] = V * pbar * dN[1]
        F[a][2] = V * pbar * dN[2]
        F[a][3] = -V / 4 * sum(taus) * dN[0] * (rho + q)
    return np.array([[float(x) for x in row] for row in F])


def shear_inputs(s, q):
    X = ref_tet(s)
    U = np.zeros((4, 4))
    U[:, 0] = X[:, 1]          # u = y
    U[:, 1] = 1.0              # v = 1
    U[:, 3] = q * X[:, 0]      # p = q x
    return X, U


@pytest.mark.parametrize("rho,mu,s,q", [(1.0, 1e-2, 1.0, 0.0), (2.5, 0.3, 0.37, -1.7),
                                        (0.8, 1e-4, 3.0, 0.5), (1.0, 1e-2, 1e-2, 2.0)])
def test_closed_form_shear_tet(rho, mu, s, q):
    X, U = shear_inputs(s, q)
    F = oracle.element(X, U, rho, mu)
    ref = closed_form_shear(rho, mu, s, q)
    scale = np.abs(ref).max()
    assert np.abs(F - ref).max() <= 1e-14 * scale


def closed_form_pressure_only(mu, s, k):
    """u = 0, p = 1 at node k (k = 1, 2, 3): grad p = e_k / s along axis k-1,
    p_bar = 1/4, tau = h^2/(c1 mu); F_a,i = V/4 dN_a/dx_i,
    F_a,4 = -(V/4) * 4 tau dN_a . grad p."""
    sd = D(s)
    V, tau = sd ** 3 / 6, sd ** 2 / (4 * D(mu))
    F = [[D(0)] * 4 for _ in range(4)]
    for a in range(4):
        dN = [D(c) / sd for c in REF_DN[a]]
        for i in range(3):
            F[a][i] = V / 4 * dN[i]
        F[a][3] = -V * tau * dN[k - 1] / sd
    return np.array([[float(x) for x in row] for row in F])


@pytest.mark.parametrize("k", [1, 2, 3])
@pytest.mark.parametrize("mu,s", [(1e-2, 1.0), (0.7, 0.25)])
def test_closed_form_pressure_only(mu, s, k):
    X = ref_tet(s)
    U = np.zeros((4, 4))
    U[k, 3] = 1.0
    F = oracle.element(X, U, 1.0, mu)
    ref = closed_form_pressure_only(mu, s, k)
    assert np.abs(F - ref).max() <= 1e-14 * np.abs(ref).max()


def test_closed_form_viscous_linear_velocity():
    """rho = 0, u_x = y: only the viscous term survives:
    F_0,x = +mu/6, F_2,x = -mu/6 on the unit reference tet."""
    mu = 1e-2
    X = ref_tet()
    U = np.zeros((4, 4))
    U[:, 0] = X[:, 1]
    F = oracle.element(X, U, 0.0, mu)
    exp = np.zeros((4, 4))
    exp[0, 0], exp[2, 0] = mu / 6, -mu / 6
    assert np.abs(F - exp).max() < 1e-17


@pytest.mark.parametrize("s,cv,rho", [(1.0, 0.07, 1.0), (0.2, 0.1, 2.0)])
def test_closed_form_vreman(s, cv, rho):
    """u = (y, x, 0): alpha has entries alpha_12 = alpha_21 = 1, so
    beta = h^2 diag(1, 1, 0), B = h^4, A = 2 and nu_t = c h^2 / sqrt(2)."""
    mu = 1e-3
    X = ref_tet(s)
    U = np.zeros((4, 4))
    U[:, 0] = X[:, 1]
    U[:, 1] = X[:, 0]
    F = oracle.element(X, U, rho, mu, c_vreman=cv, terms=oracle.T_VISC)
    mu_eff = mu + rho * cv * s * s / np.sqrt(2.0)
    V = s ** 3 / 6
    dN = np.array(REF_DN, float) / s
    exp = np.zeros((4, 4))
    exp[:, 0] = -V * mu_eff * dN[:, 1]
    exp[:, 1] = -V * mu_eff * dN[:, 0]
    assert np.abs(F - exp).max() <= 1e-14 * np.abs(exp).max()
    # pure shear has no Vreman viscosity (B = 0)
    U2 = np.zeros((4, 4))
    U2[:, 0] = X[:, 1]
    F2 = oracle.element(X, U2, rho, mu, c_vreman=cv, terms=oracle.T_VISC)
    assert np.abs(F2[:, 0] + V * mu * dN[:, 1]).max() <= 1e-15 * V * mu / s


def closed_form_vreman_stabilised(rho, mu, cv, s, q, tau_elem, c1=4, c2=2):
    """Every term with the Vreman model on, tet X0 = 0, Xk = s e_k;
    u = (y, x, 1), p = q x. grad u has du/dy = dv/dx = 1, so alpha = (grad u)^T
    has alpha_12 = alpha_21 = 1, beta = h^2 diag(1, 1, 0), B = h^4, A = 2 and
    nu_t = cv h^2 / sqrt(2): mu_eff = mu + rho cv h^2 / sqrt(2) enters the
    viscous term and tau (Sec. V-B: the element's eddy viscosity feeds its
    terms). h = s, V = s^3/6, grad N_a = e/s, div u = 0.
    Gauss point g: x_g = s N_1(xi_g), y_g = s N_2(xi_g), u_g = (y_g, x_g, 1),
    (u.grad)u = (x_g, y_g, 0), residual r_g = (rho x_g + q, rho y_g, 0).
    Galerkin convection: -rho int N_a c with c = (x, y, 0) linear, i.e. the
    consistent mass matrix V (1 + delta_ab)/20 applied to c at the nodes
    (0, (s,0,0), (0,s,0), 0). Per-element tau: |mean nodal u| = |(s/4, s/4, 1)|."""
    rho, mu, cv, s, q = D(rho), D(mu), D(cv), D(s), D(q)
    V, h, pbar = s ** 3 / 6, s, q * s / 4
    mu_eff = mu + rho * cv * h * h / D(2).sqrt()
    N = [[(QA if a == g else QB) for a in range(4)] for g in range(4)]
    xs = [s * N[g][1] for g in range(4)]
    ys = [s * N[g][2] for g in range(4)]
    if tau_elem:
        te = 1 / (c1 * mu_eff / h ** 2 + c2 * rho * (2 * (s / 4) ** 2 + 1).sqrt() / h)
        taus = [te] * 4
    else:
        taus = [1 / (c1 * mu_eff / h ** 2 + c2 * rho * (ys[g] ** 2 + xs[g] ** 2 + 1).sqrt() / h)
                for g in range(4)]
    cnode = [(D(0), D(0)), (s, D(0)), (D(0), s), (D(0), D(0))]
    F = [[D(0)] * 4 for _ in range(4)]
    for a in range(4):
        dN = [D(c) / s for c in REF_DN[a]]
        conv = [-rho * sum(V * (1 + (a == b)) / 20 * cnode[b][i] for b in range(4))
                for i in range(2)]
        adv = [ys[g] * dN[0] + xs[g] * dN[1] + dN[2] for g in range(4)]   # u_g . grad N_a
        r = [(rho * xs[g] + q, rho * ys[g]) for g in range(4)]
        supg = [-V / 4 * sum(taus[g] * rho * adv[g] * r[g][i] for g in range(4)) for i in range(2)]
        F[a][0] = conv[0] - V * mu_eff * dN[1] + V * pbar * dN[0] + supg[0]
        F[a][1] = conv[1] - V * mu_eff * dN[0] + V * pbar * dN[1] + supg[1]
        F[a][2] = V * pbar * dN[2]
        F[a][3] = -V / 4 * sum(taus[g] * (dN[0] * r[g][0] + dN[1] * r[g][1]) for g in range(4))
    return np.array([[float(x) for x in row] for row in F])


def vreman_stabilised_inputs(s, q):
    X = ref_tet(s)
    U = np.zeros((4, 4))
    U[:, 0] = X[:, 1]          # u = y
    U[:, 1] = X[:, 0]          # v = x
    U[:, 2] = 1.0              # w = 1
    U[:, 3] = q * X[:, 0]      # p = q x
    return X, U


@pytest.mark.parametrize("tau_elem", [False, True])
@pytest.mark.parametrize("rho,mu,cv,s,q", [(1.0, 1e-2, 0.07, 1.0, 0.0),
                                           (2.0, 1e-3, 0.1, 0.2, -1.3),
                                           (0.7, 5e-4, 0.07, 2.5, 0.8)])
def test_closed_form_vreman_feeds_tau(rho, mu, cv, s, q, tau_elem):
    """mu_eff (not mu) in tau and in the viscous term, with every term on and
    both tau modes; the eddy viscosity is a sizeable part of mu_eff here."""
    X, U = vreman_stabilised_inputs(s, q)
    F = oracle.element(X, U, rho, mu, c_vreman=cv, tau_elem=tau_elem)
    ref = closed_form_vreman_stabilised(rho, mu, cv, s, q, tau_elem)
    assert np.abs(F - ref).max() <= 1e-14 * np.abs(ref).max()
    # the same with the model off differs (so the check above sees mu_eff)
    ref0 = closed_form_vreman_stabilised(rho, mu, 0.0, s, q, tau_elem)
    assert np.abs(ref0 - ref).max() > 1e-6 * np.abs(ref).max()


# grad u with every beta_ij of the Vreman model nonzero:
# beta = h^2 G G^T = h^2 [[5, 2, 2], [2, 10, 3], [2, 3, 5]], whose principal
# 2x2 minors are 46, 21 and 41, so B = 108 h^4; A = sum G_ij^2 = 20.
G3 = np.array([[1.0, 2.0, 0.0], [0.0, 1.0, 3.0], [2.0, 0.0, 1.0]])
G3_B_OVER_H4, G3_A = 108, 20


@pytest.mark.parametrize("s,cv,rho", [(1.0, 0.07, 1.0), (0.3, 0.1, 2.0)])
def test_closed_form_vreman_full_3d(s, cv, rho):
    """u = G3 x + (0.5, -1, 2) on the reference tet scaled by s, viscous term
    only: F_a,i = -V mu_eff sum_j dN_a/dx_j G_ij with
    mu_eff = mu + rho cv h^2 sqrt(108/20), h = s (50-digit evaluation)."""
    mu = 1e-3
    X = ref_tet(s)
    U = np.zeros((4, 4))
    U[:, :3] = X @ G3.T + np.array([0.5, -1.0, 2.0])
    F = oracle.element(X, U, rho, mu, c_vreman=cv, terms=oracle.T_VISC)
    sd = D(s)
    mu_eff = D(mu) + D(rho) * D(cv) * sd * sd * (D(G3_B_OVER_H4) / D(G3_A)).sqrt()
    V = sd ** 3 / 6
    exp = np.zeros((4, 4))
    for a in range(4):
        dN = [D(c) / sd for c in REF_DN[a]]
        for i in range(3):
            exp[a, i] = float(-V * mu_eff * sum(dN[j] * D(G3[i, j]) for j in range(3)))
    assert np.abs(F - exp).max() <= 1e-14 * np.abs(exp).max()


def test_vreman_full_3d_on_a_general_tet():
    """The same velocity gradient on a general tet: the viscous term is
    -V mu_eff grad N G^T with grad N from an independent linear solve and
    mu_eff = mu + rho cv h^2 sqrt(108/20), h = detJ^(1/3)."""
    rng = np.random.default_rng(11)
    X = random_tet(rng)
    U = np.zeros((4, 4))
    U[:, :3] = X @ G3.T
    U[:, 3] = rng.normal(size=4)
    rho, mu, cv = 1.4, 2e-3, 0.07
    det = np.linalg.det((X[1:] - X[0]).T)
    h = np.cbrt(det)
    mu_eff = mu + rho * cv * h * h * np.sqrt(G3_B_OVER_H4 / G3_A)
    exp = -(det / 6) * mu_eff * bary_grad(X) @ G3.T
    F = oracle.element(X, U, rho, mu, c_vreman=cv, terms=oracle.T_VISC)
    assert np.abs(F[:, :3] - exp).max() <= 1e-13 * np.abs(exp).max()


def random_tet(rng):
    while True:
        X = rng.normal(size=(4, 3))
        e = X[1:] - X[0]
        if np.linalg.det(e.T) > 0.2:
            return X


def bary_grad(X):
    """Gradients of barycentric coordinates by an independent linear solve:
    [1 x y z] c = delta -> grad N_a = c[1:, a]."""
    A = np.hstack([np.ones((4, 1)), X])
    C = np.linalg.solve(A, np.eye(4))
    return C[1:].T  # [a][j]


@pytest.mark.parametrize("seed", range(5))
def test_term_invariants_random_tets(seed):
    rng = np.random.default_rng(100 + seed)
    X = random_tet(rng)
    U = rng.normal(size=(4, 4))
    rho, mu = 1.3, 0.05
    dN = bary_grad(X)
    V = abs(np.linalg.det((X[1:] - X[0]).T)) / 6
    G = U[:, :3].T @ dN           # G[i][j] = du_i/dx_j
    div = np.trace(G)
    Fs = {t: oracle.element(X, U, rho, mu, c_vreman=0.0, terms=t)
          for t in (oracle.T_CONV, oracle.T_VISC, oracle.T_PRES, oracle.T_SUPG, oracle.T_CONT,
                    oracle.T_PSPG)}
    tol = 1e-13 * (1 + np.abs(U).max()) ** 2
    # sum_a grad N_a = 0: these terms sum to zero over the element's nodes
    for t in (oracle.T_VISC, oracle.T_PRES, oracle.T_SUPG, oracle.T_PSPG):
        assert np.abs(Fs[t].sum(axis=0)).max() < tol
    # Galerkin continuity sums to -V div u
    assert abs(Fs[oracle.T_CONT][:, 3].sum() + V * div) < tol
    # term supports: momentum terms leave column 4 alone and vice versa
    for t in (oracle.T_CONV, oracle.T_VISC, oracle.T_PRES, oracle.T_SUPG):
        assert np.all(Fs[t][:, 3] == 0)
    for t in (oracle.T_CONT, oracle.T_PSPG):
        assert np.all(Fs[t][:, :3] == 0)
    # textbook forms from the independent gradients
    M = V * (np.ones((4, 4)) + np.eye(4)) / 20.0          # P1 consistent mass matrix
    conv = -rho * M @ (U[:, :3] @ G.T)                    # -rho sum_b M_ab (G u_b)
    assert np.abs(Fs[oracle.T_CONV][:, :3] - conv).max() < tol
    visc = -V * mu * dN @ G.T                             # -V mu G grad N_a
    assert np.abs(Fs[oracle.T_VISC][:, :3] - visc).max() < tol
    pres = V * U[:, 3].mean() * dN                        # V p_bar grad N_a
    assert np.abs(Fs[oracle.T_PRES][:, :3] - pres).max() < tol
    assert np.abs(Fs[oracle.T_CONT][:, 3] + V * div / 4).max() < tol
    # the full RHS is the sum of its terms
    full = oracle.element(X, U, rho, mu)
    assert np.abs(full - sum(Fs.values())).max() < tol


def test_element_even_permutation_and_rigid_motion():
    rng = np.random.default_rng(7)
    X = random_tet(rng)
    U = rng.normal(size=(4, 4))
    for cv in (0.0, 0.07):
        F = oracle.element(X, U, 1.0, 1e-2, c_vreman=cv)
        for perm in ([1, 2, 0, 3], [2, 0, 1, 3], [1, 0, 3, 2], [3, 2, 1, 0], [0, 2, 3, 1]):
            Fp = oracle.element(X[perm], U[perm], 1.0, 1e-2, c_vreman=cv)
            assert np.abs(Fp - F[perm]).max() < 1e-13 * np.abs(F).max()
        # rotation + translation: momentum rotates, continuity invariant
        Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
        if np.linalg.det(Q) < 0:
            Q[:, 0] *= -1
        Xr = X @ Q.T + np.array([0.3, -1.2, 2.0])
        Ur = U.copy()
        Ur[:, :3] = U[:, :3] @ Q.T
        Fr = oracle.element(Xr, Ur, 1.0, 1e-2, c_vreman=cv)
        assert np.abs(Fr[:, :3] - F[:, :3] @ Q.T).max() < 1e-12 * np.abs(F).max()
        assert np.abs(Fr[:, 3] - F[:, 3]).max() < 1e-12 * np.abs(F).max()


def test_linearity_in_pressure():
    rng = np.random.default_rng(3)
    X = random_tet(rng)
    U = rng.normal(size=(4, 4))
    p1, p2 = rng.normal(size=4), rng.normal(size=4)

    def f(p):
        W = U.copy()
        W[:, 3] = p
        return oracle.element(X, W, 1.0, 1e-2, c_vreman=0.07)
    d = f(p1 + p2) - f(p1) - f(p2) + f(np.zeros(4))
    assert np.abs(d).max() < 1e-13 * np.abs(f(p1)).max()


def test_inverted_tet_rejected():
    X = ref_tet()[[0, 2, 1, 3]]
    with pytest.raises(ValueError):
        oracle.element(X, np.zeros((4, 4)), 1.0, 1e-2)


@pytest.fixture(scope="module")
def mesh6():
    coords, conn, _, _ = mg.box_mesh(6, 0.1)
    up = mg.fields(coords)
    return coords, conn, up


def boundary_faces(conn):
    f = np.concatenate([conn[[1, 2, 3]], conn[[0, 2, 3]], conn[[0, 1, 3]], conn[[0, 1, 2]]], axis=1)
    fs = np.sort(f.T, axis=1)
    uf, counts = np.unique(fs, axis=0, return_counts=True)
    return uf[counts == 1]


def outward_area_normals(coords, faces):
    P = coords[:, faces]  # [3][F][3]
    n = np.cross((P[:, :, 1] - P[:, :, 0]).T, (P[:, :, 2] - P[:, :, 0]).T) / 2.0  # [F][3]
    centre = P.mean(axis=2).T
    sign = np.sign(np.sum(n * (centre - 0.5), axis=1))
    return n * sign[:, None]


def test_global_divergence_theorem(mesh6):
    """sum over nodes of the continuity RHS = -int div u = -oint u.n
    (the stabilisation part sums to zero element by element)."""
    coords, conn, up = mesh6
    rhs = oracle.assemble(coords, conn, up, 1.0, 1e-2)
    faces = boundary_faces(conn)
    nA = outward_area_normals(coords, faces)
    umean = up[:3, faces].mean(axis=2).T            # [F][3]
    flux = np.sum(nA * umean)
    assert abs(rhs[3].sum() + flux) < 1e-13 * (1 + abs(flux))


def test_constant_fields(mesh6):
    coords, conn, _ = mesh6
    N = coords.shape[1]
    # constant velocity, zero pressure: no gradients, no residual -> RHS = 0
    up = np.zeros((4, N))
    up[:3] = np.array([0.3, -2.0, 1.1])[:, None]
    rhs = oracle.assemble(coords, conn, up, 1.0, 1e-2, c_vreman=0.07)
    assert np.abs(rhs).max() < 1e-16
    # zero velocity, constant pressure p0: momentum RHS = p0 oint N_a n
    # (zero at interior nodes), continuity RHS = 0
    p0 = 1.7
    up = np.zeros((4, N))
    up[3] = p0
    rhs = oracle.assemble(coords, conn, up, 1.0, 1e-2)
    faces = boundary_faces(conn)
    nA = outward_area_normals(coords, faces)
    expect = np.zeros((3, N))
    for k in range(3):
        np.add.at(expect.T, faces[:, k], p0 * nA / 3.0)
    assert np.abs(rhs[:3] - expect).max() < 1e-15
    assert np.abs(rhs[3]).max() < 1e-16


def test_global_invariances(mesh6):
    coords, conn, up = mesh6
    N, E = coords.shape[1], conn.shape[1]
    rhs = oracle.assemble(coords, conn, up, 1.0, 1e-2, c_vreman=0.07)
    scale = np.abs(rhs).max()
    # node renumbering
    order = mg.random_order(N)
    c2, cn2, up2 = mg.renumber(order, coords, conn, up)
    rhs2 = oracle.assemble(c2, cn2, up2, 1.0, 1e-2, c_vreman=0.07)
    assert np.abs(rhs2 - rhs[:, order]).max() < 1e-14 * scale
    # element order
    perm = np.random.default_rng(0).permutation(E)
    rhs3 = oracle.assemble(coords, conn[:, perm], up, 1.0, 1e-2, c_vreman=0.07)
    assert np.abs(rhs3 - rhs).max() < 1e-14 * scale
    # element slices add up
    half = oracle.assemble(coords, conn, up, 1.0, 1e-2, c_vreman=0.07, e0=0, e1=E // 3)
    rest = oracle.assemble(coords, conn, up, 1.0, 1e-2, c_vreman=0.07, e0=E // 3, e1=E)
    assert np.abs(half + rest - rhs).max() < 1e-14 * scale
    # rigid rotation of the whole problem
    Q, _ = np.linalg.qr(np.random.default_rng(1).normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    upr = up.copy()
    upr[:3] = Q @ up[:3]
    rr = oracle.assemble(Q @ coords, conn, upr, 1.0, 1e-2, c_vreman=0.07)
    assert np.abs(rr[:3] - Q @ rhs[:3]).max() < 1e-13 * scale
    assert np.abs(rr[3] - rhs[3]).max() < 1e-13 * scale


def test_complex_step_matches_central_differences(mesh6):
    coords, conn, up = mesh6
    d = mg.normal(up.shape, seed=mg.SEED_DIRS)
    for cv in (0.0, 0.07):
        s = 1e-30
        jv = oracle.assemble_complex(coords, conn, up + 1j * s * d, 1.0, 1e-2, c_vreman=cv).imag / s
        eps = 1e-6
        fd = (oracle.assemble(coords, conn, up + eps * d, 1.0, 1e-2, c_vreman=cv) -
              oracle.assemble(coords, conn, up - eps * d, 1.0, 1e-2, c_vreman=cv)) / (2 * eps)
        assert np.linalg.norm(jv - fd) <= 1e-7 * np.linalg.norm(jv)
        # the complex evaluation's real part is the real RHS
        re = oracle.assemble_complex(coords, conn, up + 1j * s * d, 1.0, 1e-2, c_vreman=cv).real
        assert np.abs(re - oracle.assemble(coords, conn, up, 1.0, 1e-2, c_vreman=cv)).max() < 1e-15


def test_vjp_against_full_complex_step_jacobian():
    coords, conn, _, _ = mg.box_mesh(2, 0.1)
    up = mg.fields(coords)
    N = coords.shape[1]
    w = mg.normal((4, N), seed=mg.SEED_COT)
    for cv in (0.0, 0.07):
        s = 1e-30
        J = np.empty((4 * N, 4 * N))
        for col in range(4 * N):
            e = np.zeros(4 * N)
            e[col] = s
            J[:, col] = (oracle.assemble_complex(coords, conn, up + 1j * e.reshape(4, N), 1.0,
                                                 1e-2, c_vreman=cv).imag / s).ravel()
        ref = (J.T @ w.ravel()).reshape(4, N)
        g = oracle.vjp(coords, conn, up, w, 1.0, 1e-2, c_vreman=cv)
        assert np.linalg.norm(g - ref) <= 1e-13 * np.linalg.norm(ref)


def test_vjp_dot_product_identity(mesh6):
    coords, conn, up = mesh6
    N = coords.shape[1]
    w = mg.normal((4, N), seed=mg.SEED_COT)
    v = mg.normal((4, N), seed=mg.SEED_DIRS)
    s = 1e-30
    jv = oracle.assemble_complex(coords, conn, up + 1j * s * v, 1.0, 1e-4).imag / s
    g = oracle.vjp(coords, conn, up, w, 1.0, 1e-4)
    lhs, rhs = np.sum(w * jv), np.sum(g * v)
    assert abs(lhs - rhs) <= 1e-12 * np.sqrt(np.sum(w * w) * np.sum(jv * jv))


# ---- formulation variants: skew-symmetric convection, per-element tau ----

def closed_form_shear_variants(rho, mu, s, q, skew, tau_elem, c1=4, c2=2):
    """As closed_form_shear, with the variants: the skew-symmetric Galerkin
    convection -rho/2 int[N_a (u.grad)u_i - (u.grad N_a) u_i] (u.grad N_a at
    Gauss point g: y_g dN_a/dx + dN_a/dy) and/or one tau from the mean
    velocity (s/4, 1, 0)."""
    rho, mu, s, q = D(rho), D(mu), D(s), D(q)
    V, h, pbar = s ** 3 / 6, s, q * s / 4
    ys = [s * (QA if g == 2 else QB) for g in range(4)]
    Ng = [[(QA if a == g else QB) for a in range(4)] for g in range(4)]
    if tau_elem:
        te = 1 / (c1 * mu / h ** 2 + c2 * rho * ((s / 4) ** 2 + 1).sqrt() / h)
        taus = [te] * 4
    else:
        taus = [1 / (c1 * mu / h ** 2 + c2 * rho * (y * y + 1).sqrt() / h) for y in ys]
    F = [[D(0)] * 4 for _ in range(4)]
    for a in range(4):
        dN = [D(c) / s for c in REF_DN[a]]
        adv = [ys[g] * dN[0] + dN[1] for g in range(4)]       # u_g . grad N_a
        if skew:
            conv_x = -rho / 2 * sum(V / 4 * (Ng[g][a] * 1 - adv[g] * ys[g]) for g in range(4))
            conv_y = -rho / 2 * sum(V / 4 * (0 - adv[g] * 1) for g in range(4))
        else:
            conv_x, conv_y = -V * rho / 4, D(0)
        supg = sum(taus[g] * rho * adv[g] * (rho + q) for g in range(4))
        F[a][0] = conv_x - V * mu * dN[1] + V * pbar * dN[0] - V / 4 * supg
        F[a][1] = conv_y + V * pbar * dN[1]
        F[a][2] = V * pbar * dN[2]
        F[a][3] = -V / 4 * sum(taus) * dN[0] * (rho + q)
    return np.array([[float(x) for x in row] for row in F])


@pytest.mark.parametrize("skew,tau_elem", [(True, False), (False, True), (True, True)])
@pytest.mark.parametrize("rho,mu,s,q", [(1.0, 1e-2, 1.0, 0.0), (2.5, 0.3, 0.37, -1.7)])
def test_closed_form_shear_variants(skew, tau_elem, rho, mu, s, q):
    X, U = shear_inputs(s, q)
    F = oracle.element(X, U, rho, mu, skew=skew, tau_elem=tau_elem)
    ref = closed_form_shear_variants(rho, mu, s, q, skew, tau_elem)
    assert np.abs(F - ref).max() <= 1e-14 * np.abs(ref).max()
    # the default-form closed form is the same function with both flags off
    base = closed_form_shear_variants(rho, mu, s, q, False, False)
    assert np.abs(base - closed_form_shear(rho, mu, s, q)).max() <= 1e-15 * np.abs(base).max()


def test_skew_convection_does_no_work(mesh6):
    """Energy preservation: sum over nodes of u . F_conv = 0 for the
    skew-symmetric form (pointwise skew integrand), and not for the
    convective form."""
    coords, conn, up = mesh6
    for skew, expect_zero in ((True, True), (False, False)):
        f = oracle.assemble(coords, conn, up, 1.3, 1e-2, terms=oracle.T_CONV, skew=skew)
        work = float(np.sum(up[:3] * f[:3]))
        scale = float(np.sum(np.abs(up[:3] * f[:3])))
        if expect_zero:
            assert abs(work) <= 1e-14 * scale
        else:
            assert abs(work) > 1e-6 * scale


def test_variants_invariants_and_derivatives(mesh6):
    coords, conn, up = mesh6
    kw = dict(skew=True, tau_elem=True, c_vreman=0.07)
    rhs = oracle.assemble(coords, conn, up, 1.0, 1e-2, **kw)
    scale = np.abs(rhs).max()
    # rigid rotation
    Q, _ = np.linalg.qr(np.random.default_rng(4).normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] *= -1
    upr = up.copy()
    upr[:3] = Q @ up[:3]
    rr = oracle.assemble(Q @ coords, conn, upr, 1.0, 1e-2, **kw)
    assert np.abs(rr[:3] - Q @ rhs[:3]).max() < 1e-13 * scale
    # constant velocity u0: only the skew term's boundary flux remains,
    # rho/2 u0_i (u0 . oint N_a n dS), zero at interior nodes
    N = coords.shape[1]
    u0 = np.array([0.3, -2.0, 1.1])
    uc = np.zeros((4, N))
    uc[:3] = u0[:, None]
    got = oracle.assemble(coords, conn, uc, 1.3, 1e-2, **kw)
    faces = boundary_faces(conn)
    nA = outward_area_normals(coords, faces)
    flux = np.zeros(N)
    for k in range(3):
        np.add.at(flux, faces[:, k], nA @ u0 / 3.0)
    expect = 0.5 * 1.3 * u0[:, None] * flux[None, :]
    assert np.abs(got[:3] - expect).max() < 1e-15
    assert np.abs(got[3]).max() < 1e-16
    # complex step agrees with central differences, and the element-Jacobian VJP
    # satisfies the dot-product identity
    d = mg.normal(up.shape, seed=mg.SEED_DIRS)
    jv = oracle.assemble_complex(coords, conn, up + 1e-30j * d, 1.0, 1e-2, **kw).imag / 1e-30
    eps = 1e-6
    fd = (oracle.assemble(coords, conn, up + eps * d, 1.0, 1e-2, **kw) -
          oracle.assemble(coords, conn, up - eps * d, 1.0, 1e-2, **kw)) / (2 * eps)
    assert np.linalg.norm(jv - fd) <= 1e-7 * np.linalg.norm(jv)
    w = mg.normal(up.shape, seed=mg.SEED_COT)
    g = oracle.vjp(coords, conn, up, w, 1.0, 1e-2, **kw)
    assert abs(np.sum(w * jv) - np.sum(g * d)) <= 1e-12 * np.sqrt(np.sum(w * w) * np.sum(jv * jv))


# ---- explicit time stepping (oracle composition) ----

def test_lumped_mass_sums_to_volume(mesh6):
    coords, conn, _ = mesh6
    m = oracle.lumped_mass(coords, conn)
    assert abs(m.sum() - 1.0) < 1e-14 and (m > 0).all()
    # an interior node of the undistorted mesh carries h^3 (24 tets of h^3/6, /4 each)
    c0, cn0, _, _ = mg.box_mesh(4, 0.0)
    m0 = oracle.lumped_mass(c0, cn0)
    centre = 2 + 5 * (2 + 5 * 2)
    assert abs(m0[centre] - 0.25 ** 3) < 1e-16


@pytest.mark.parametrize("z", [-0.3, 0.5, -1.2 + 0.7j])
def test_runge_kutta_amplification(z):
    """On du/dt = lam u the schemes reproduce their amplification polynomials:
    Euler 1 + z, SSP-RK3 1 + z + z^2/2 + z^3/6 (z = lam dt)."""
    lam, dt = z / 0.1, 0.1
    u0 = np.array([1.0 + 0j, -2.0])
    L = lambda u: lam * u  # noqa: E731
    assert np.allclose(oracle.euler(u0, L, dt), (1 + z) * u0, rtol=1e-15)
    assert np.allclose(oracle.ssprk3(u0, L, dt), (1 + z + z * z / 2 + z ** 3 / 6) * u0,
                       rtol=1e-15)


def test_explicit_step_keeps_constant_velocity_and_pressure(mesh6):
    coords, conn, up = mesh6
    uc = np.zeros_like(up)
    uc[:3] = np.array([0.3, -2.0, 1.1])[:, None]
    uc[3] = up[3]  # pressure is frozen; constant velocity with variable p changes u
    out = oracle.explicit_step(coords, conn, uc, 1.0, 1e-2, 1e-3, "ssprk3")
    assert np.array_equal(out[3], uc[3])
    up0 = uc.copy()
    up0[3] = 0.0
    out0 = oracle.explicit_step(coords, conn, up0, 1.0, 1e-2, 1e-3, "ssprk3")
    assert np.abs(out0 - up0).max() < 1e-15
