"""The oracle's pins catch plausible mistakes (CPU).

Each case copies the oracle source, plants one plausible slip in it (a
dropped density, a flipped sign, a transposed gradient, a wrong element size,
a wrong Gauss weight, ...), builds it in a temporary directory and runs the
pin battery below against it: every mutant must fail at least one pin, and
the real oracle must pass them all. Nothing in the repository is modified.
"""
import importlib.util
import os
import shutil
import subprocess

import numpy as np
import pytest

import meshgen as mg
import test_oracle_pins as pins

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE_DIR = os.path.join(ROOT, "oracle")

MUTATIONS = [
    ("SUPG without density", "f += -tau * P.rho * ugradNa * r[i];", "f += -tau * ugradNa * r[i];"),
    ("pressure term sign", "f += pg * dN[a][i];", "f += -pg * dN[a][i];"),
    ("transposed gradient in (u.grad)u", "cg[i] += ug[j] * G[i][j];", "cg[i] += ug[j] * G[j][i];"),
    ("element size h = detJ", "const double h = std::cbrt(det);", "const double h = det;"),
    ("Gauss weight", "const double QA = (5.0 + 3.0 * SQRT5) / 20.0;",
     "const double QA = (5.0 + 2.0 * SQRT5) / 20.0;"),
    ("grad N_0 sign", "dN[0][j] = -(Ji[0][j] + Ji[1][j] + Ji[2][j]);",
     "dN[0][j] = (Ji[0][j] + Ji[1][j] + Ji[2][j]);"),
    ("residual without grad p", "r[i] = P.rho * cg[i] + gp[i];", "r[i] = P.rho * cg[i];"),
    ("tau without density", "P.c2 * P.rho * unorm / h);", "P.c2 * unorm / h);"),
    ("tau viscous scale h instead of h^2",
     "T tau = 1.0 / (P.c1 * mu_eff / (h * h) +", "T tau = 1.0 / (P.c1 * mu_eff / h +"),
    ("continuity sign", "f4 += -N[a] * divu;", "f4 += N[a] * divu;"),
    ("PSPG missing a component", "dN[a][0] * r[0] + dN[a][1] * r[1] + dN[a][2] * r[2]",
     "dN[a][0] * r[0] + dN[a][1] * r[1]"),
    ("viscous sign", "f += -mu_eff * gg;", "f += mu_eff * gg;"),
    ("Vreman without h^2", "be[i][j] += h * h * al[m][i] * al[m][j];",
     "be[i][j] += al[m][i] * al[m][j];"),
    ("skew convection without the 1/2", "f += -0.5 * P.rho * (N[a] * cg[i] - ugradNa * ug[i]);",
     "f += -P.rho * (N[a] * cg[i] - ugradNa * ug[i]);"),
    ("convection with a uniform weight", "f += -P.rho * N[a] * cg[i];",
     "f += -P.rho * 0.25 * cg[i];"),
    ("per-element tau from the sum, not the mean",
     "ub[i] = 0.25 * (U[0][i] + U[1][i] + U[2][i] + U[3][i]);",
     "ub[i] = (U[0][i] + U[1][i] + U[2][i] + U[3][i]);"),
    ("viscous gradient transposed", "gg += dN[a][j] * G[i][j];", "gg += dN[a][j] * G[j][i];"),
    ("Gauss-point tau with mu instead of mu_eff", "T tau = 1.0 / (P.c1 * mu_eff / (h * h) +",
     "T tau = 1.0 / (P.c1 * P.mu / (h * h) +"),
    ("per-element tau with mu instead of mu_eff", "tau_e = 1.0 / (P.c1 * mu_eff / (h * h) +",
     "tau_e = 1.0 / (P.c1 * P.mu / (h * h) +"),
    ("viscous term with mu instead of mu_eff", "f += -mu_eff * gg;", "f += -P.mu * gg;"),
    ("eddy viscosity without density", "mu_eff = P.mu + P.rho * (P.c_vreman",
     "mu_eff = P.mu + (P.c_vreman"),
    ("Vreman B without beta_13^2", "be[0][2] * be[0][2] + be[1][1]",
     "0.0 * be[0][2] + be[1][1]"),
    ("Vreman B without beta_23^2", "be[1][1] * be[2][2] - be[1][2] * be[1][2];",
     "be[1][1] * be[2][2];"),
    ("Vreman A from the diagonal only", "A += al[i][j] * al[i][j];", "A += al[i][i] * al[i][i] / 3.0;"),
]


def load_oracle(lib_path, tag):
    """A fresh copy of the oracle package bound to the library at lib_path."""
    spec = importlib.util.spec_from_file_location(f"oracle_{tag}",
                                                  os.path.join(ORACLE_DIR, "__init__.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod._lib = None
    mod.build = lambda force=False: lib_path
    return mod


def battery(o):
    """The fast pins of test_oracle_pins, run against oracle-like module o.
    Returns the names of the pins that fail."""
    failed = []

    def check(name, ok):
        if not ok:
            failed.append(name)

    try:
        for rho, mu, s, q in [(1.0, 1e-2, 1.0, 0.0), (2.5, 0.3, 0.37, -1.7)]:
            X, U = pins.shear_inputs(s, q)
            ref = pins.closed_form_shear(rho, mu, s, q)
            check("shear closed form", np.abs(o.element(X, U, rho, mu) - ref).max()
                  <= 1e-14 * np.abs(ref).max())
            for skew, te in ((True, False), (False, True)):
                refv = pins.closed_form_shear_variants(rho, mu, s, q, skew, te)
                got = o.element(X, U, rho, mu, skew=skew, tau_elem=te)
                check("variant closed form", np.abs(got - refv).max() <= 1e-14 * np.abs(refv).max())
        # pressure-only closed form along every axis (PSPG components)
        for k in (1, 2, 3):
            U = np.zeros((4, 4))
            U[k, 3] = 1.0
            ref = pins.closed_form_pressure_only(0.7, 0.25, k)
            check("pressure-only closed form", np.abs(o.element(pins.ref_tet(0.25), U, 1.0, 0.7) - ref
                                                       ).max() <= 1e-14 * np.abs(ref).max())
        # Vreman closed form
        s, cv, rho, mu = 0.2, 0.1, 2.0, 1e-3
        X = pins.ref_tet(s)
        U = np.zeros((4, 4))
        U[:, 0], U[:, 1] = X[:, 1], X[:, 0]
        F = o.element(X, U, rho, mu, c_vreman=cv, terms=o.T_VISC)
        mu_eff = mu + rho * cv * s * s / np.sqrt(2.0)
        dN = np.array(pins.REF_DN, float) / s
        exp = np.zeros((4, 4))
        exp[:, 0] = -(s ** 3 / 6) * mu_eff * dN[:, 1]
        exp[:, 1] = -(s ** 3 / 6) * mu_eff * dN[:, 0]
        check("vreman closed form", np.abs(F - exp).max() <= 1e-14 * np.abs(exp).max())
        # Vreman with every term on: mu_eff in tau, both tau modes
        for te in (False, True):
            X, U = pins.vreman_stabilised_inputs(0.2, -1.3)
            ref = pins.closed_form_vreman_stabilised(2.0, 1e-3, 0.1, 0.2, -1.3, te)
            got = o.element(X, U, 2.0, 1e-3, c_vreman=0.1, tau_elem=te)
            check("vreman stabilised closed form", np.abs(got - ref).max()
                  <= 1e-14 * np.abs(ref).max())
        # Vreman with every beta_ij nonzero
        s3 = 0.3
        X = pins.ref_tet(s3)
        U = np.zeros((4, 4))
        U[:, :3] = X @ pins.G3.T
        F = o.element(X, U, 2.0, 1e-3, c_vreman=0.1, terms=o.T_VISC)
        mu_eff = 1e-3 + 2.0 * 0.1 * s3 * s3 * np.sqrt(pins.G3_B_OVER_H4 / pins.G3_A)
        exp = -(s3 ** 3 / 6) * mu_eff * (np.array(pins.REF_DN, float) / s3) @ pins.G3.T
        check("vreman 3-d closed form", np.abs(F[:, :3] - exp).max() <= 1e-13 * np.abs(exp).max())
        # per-term textbook forms on random tets
        rng = np.random.default_rng(100)
        for _ in range(3):
            X = pins.random_tet(rng)
            U = rng.normal(size=(4, 4))
            dNr = pins.bary_grad(X)
            V = abs(np.linalg.det((X[1:] - X[0]).T)) / 6
            G = U[:, :3].T @ dNr
            M = V * (np.ones((4, 4)) + np.eye(4)) / 20.0
            tol = 1e-13 * (1 + np.abs(U).max()) ** 2
            check("consistent-mass convection", np.abs(
                o.element(X, U, 1.3, 0.05, terms=o.T_CONV)[:, :3] + 1.3 * M @ (U[:, :3] @ G.T)
            ).max() < tol)
            check("viscous textbook", np.abs(
                o.element(X, U, 1.3, 0.05, terms=o.T_VISC)[:, :3] + V * 0.05 * dNr @ G.T
            ).max() < tol)
            check("pressure textbook", np.abs(
                o.element(X, U, 1.3, 0.05, terms=o.T_PRES)[:, :3] - V * U[:, 3].mean() * dNr
            ).max() < tol)
            check("continuity textbook", np.abs(
                o.element(X, U, 1.3, 0.05, terms=o.T_CONT)[:, 3] + V * np.trace(G) / 4).max() < tol)
            for t in (o.T_VISC, o.T_PRES, o.T_SUPG, o.T_PSPG):
                check("sum over nodes", np.abs(o.element(X, U, 1.3, 0.05, terms=t).sum(axis=0)).max()
                      < tol)
        # skew convection does no work on a small mesh
        coords, conn, _, _ = mg.box_mesh(3, 0.1)
        up = mg.fields(coords)
        f = o.assemble(coords, conn, up, 1.3, 1e-2, terms=o.T_CONV, skew=True)
        check("skew zero work", abs(np.sum(up[:3] * f[:3])) <= 1e-14 * np.sum(np.abs(up[:3] * f[:3])))
    except Exception as exc:  # a mutant that crashes a check fails it
        failed.append(f"exception {exc!r}")
    return failed


def build_variant(src_text, out_dir, tag):
    src = os.path.join(out_dir, f"oracle_{tag}.cpp")
    lib = os.path.join(out_dir, f"liboracle_{tag}.so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.check_call(["g++", "-O1", "-std=c++17", "-shared", "-fPIC", "-o", lib, src])
    return lib


@pytest.fixture(scope="module")
def source():
    with open(os.path.join(ORACLE_DIR, "nsrhs_oracle.cpp")) as f:
        return f.read()


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_real_oracle_passes_the_battery(source, tmp_path):
    o = load_oracle(build_variant(source, str(tmp_path), "real"), "real")
    assert battery(o) == []


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(source, tmp_path, name, old, new):
    assert source.count(old) >= 1, f"mutation site not found: {old}"
    mutant = source.replace(old, new)
    o = load_oracle(build_variant(mutant, str(tmp_path), "m"), "m")
    failed = battery(o)
    assert failed, f"planted mistake '{name}' passed every pin"
