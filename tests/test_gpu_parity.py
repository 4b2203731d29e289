"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Tolerances (written here, from the stated requirements):
  * FP64 form: norm-wise relative error <= 1e-12 over the full [4][N] RHS
    (atomic summation order is the only allowed difference), and every
    entry within 1e-12 * max|RHS|;
  * mixed form: norm-wise relative error <= 1e-5;
  * adjoint: <= 1e-12 against the oracle's complex-step element Jacobians,
    <= 1e-6 against central finite differences (step 1e-6).
"""
import numpy as np
import pytest
import torch

import meshgen as mg
import oracle
import paper_2403_08777_gb300 as ns
from paper_2403_08777_gb300 import _abi

pytestmark = pytest.mark.gpu

TOL_FP64 = 1e-12
TOL_MIXED = 1e-5
TOL_VJP_ORACLE = 1e-12
TOL_VJP_FD = 1e-6


@pytest.fixture(scope="module")
def dev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ns.load_library()
    return torch.device("cuda:0")


def relerr(x, ref):
    return float(np.linalg.norm(x - ref) / np.linalg.norm(ref))


def on_dev(dev, *arrays):
    return [torch.from_numpy(np.ascontiguousarray(a)).to(dev) for a in arrays]


def gpu_rhs(dev, w, params=None, mesh=None, up=None):
    coords, conn, up_d = on_dev(dev, w.coords, w.conn, w.up if up is None else up)
    mesh = mesh or ns.Mesh(coords, conn)
    p = params or ns.Params(rho=w.rho, mu=w.mu, c_vreman=w.c_vreman)
    if p.precision == "mixed":
        up_d = up_d.float()
    return mesh.assemble(up_d, p).cpu().numpy(), mesh


def check_fp64(x, ref):
    assert relerr(x, ref) <= TOL_FP64, relerr(x, ref)
    assert np.abs(x - ref).max() <= TOL_FP64 * np.abs(ref).max()


FWD_CASES = [
    # n, jitter, order, mu, mag_max, c_vreman
    (8, 0.1, "lex", 1e-2, 0.0, 0.0),       # the 8^3 parity mesh
    (8, 0.1, "lex", 1e-2, 0.0, 0.07),
    (13, 0.1, "random", 1e-2, 0.0, 0.0),   # E = 13182: ragged against every block size
    (24, 0.1, "rcm", 1e-4, 10.0, 0.0),     # paper-scale settings, small mesh
    (24, 0.3, "rcm", 1e-4, 10.0, 0.07),
    (40, 0.1, "random", 1e-2, 0.0, 0.0),   # several waves of blocks
]


@pytest.mark.parametrize("n,jitter,order,mu,mag,cv", FWD_CASES)
def test_fp64_forward_matches_oracle(dev, n, jitter, order, mu, mag, cv):
    w = mg.make_workload(n, jitter=jitter, order=order, mu=mu, mag_max=mag, c_vreman=cv)
    ref = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu, c_vreman=cv)
    for scatter in ("auto", "atomic", "block"):
        x, mesh = gpu_rhs(dev, w, ns.Params(rho=w.rho, mu=w.mu, c_vreman=cv, scatter=scatter))
        check_fp64(x, ref)
        info = mesh.info()
        assert info["n_blocks"] == (w.n_elems + 255) // 256 and info["block_elems"] == 256
        mesh.close()


def test_fp64_forward_64cube_and_renumbering(dev):
    """64^3 (1.57M tets): lexicographic, random and RCM orders all match the
    oracle, and agree with each other after undoing the permutation."""
    base = mg.make_workload(64)
    ref = oracle.assemble(base.coords, base.conn, base.up, base.rho, base.mu)
    x, m = gpu_rhs(dev, base)
    check_fp64(x, ref)
    m.close()
    for order in (mg.random_order(base.n_nodes), mg.rcm_order(base.conn, base.n_nodes)):
        c2, cn2, up2 = mg.renumber(order, base.coords, base.conn, base.up)
        w2 = mg.Workload("perm", 64, c2, cn2, up2, base.rho, base.mu)
        x2, m2 = gpu_rhs(dev, w2)
        check_fp64(x2, ref[:, order])
        m2.close()


def test_ragged_element_counts(dev):
    """Meshes of 1, 31, 127, 128, 129 and 1000 elements (prefixes of a mesh,
    with nodes left unused)."""
    w = mg.make_workload(6, jitter=0.2, order="random")
    for E in (1, 31, 127, 128, 129, 255, 256, 257, 1000):
        sub = mg.Workload("sub", 6, w.coords, np.ascontiguousarray(w.conn[:, :E]), w.up, 1.0, 1e-2)
        ref = oracle.assemble(sub.coords, sub.conn, sub.up, 1.0, 1e-2)
        for scatter in ("atomic", "block"):
            x, m = gpu_rhs(dev, sub, ns.Params(rho=1.0, mu=1e-2, scatter=scatter))
            check_fp64(x, ref)
            m.close()
            x, m = gpu_rhs(dev, sub, ns.Params(rho=1.0, mu=1e-2, scatter=scatter,
                                                precision="mixed"))
            assert relerr(x, ref) <= TOL_MIXED
            m.close()


def test_block_scatter_on_disconnected_elements(dev):
    """600 tets that share no node: every block touches 1024 distinct nodes,
    the largest staging capacity. FP64 forward and the mixed forward and
    adjoint on the block scatter match the oracle; the FP64 adjoint's block
    stages do not fit one CTA there, which the call reports."""
    rng = np.random.default_rng(21)
    E = 600
    base = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float) * 0.1
    X = base[None, :, :] + rng.uniform(-0.5, 0.5, size=(E, 1, 3)) + rng.uniform(-0.01, 0.01, (E, 4, 3))
    coords = np.ascontiguousarray(X.reshape(-1, 3).T)
    conn = np.ascontiguousarray(np.arange(4 * E, dtype=np.int32).reshape(E, 4).T)
    up = rng.normal(size=(4, 4 * E))
    w = mg.Workload("disjoint", 1, coords, conn, up, 1.0, 1e-2)
    ref = oracle.assemble(coords, conn, up, 1.0, 1e-2)
    cot = mg.normal((4, 4 * E), seed=mg.SEED_COT)
    gref = oracle.vjp(coords, conn, up, cot, 1.0, 1e-2)
    c_d, n_d, up_d, cot_d = on_dev(dev, coords, conn, up, cot)
    m = ns.Mesh(c_d, n_d)
    check_fp64(m.assemble(up_d, ns.Params(scatter="block")).cpu().numpy(), ref)
    pm = ns.Params(scatter="block", precision="mixed")
    assert relerr(m.assemble(up_d.float(), pm).cpu().numpy(), ref) <= TOL_MIXED
    assert relerr(m.assemble_vjp(up_d.float(), cot_d.float(), pm).cpu().numpy(), gref) <= 1e-6
    with pytest.raises(_abi.NSRHSError):
        m.assemble_vjp(up_d, cot_d, ns.Params(scatter="block"))
    g = m.assemble_vjp(up_d, cot_d, ns.Params()).cpu().numpy()   # atomic: fine
    assert relerr(g, gref) <= TOL_VJP_ORACLE
    # the one-pass call: the mixed block stages (two entry buffers) fit, the
    # FP64 ones do not
    r1, g1 = m.assemble_rhs_vjp(up_d.float(), cot_d.float(), pm)
    assert relerr(r1.cpu().numpy(), ref) <= TOL_MIXED
    assert relerr(g1.cpu().numpy(), gref) <= 1e-6
    with pytest.raises(_abi.NSRHSError) as ei:
        m.assemble_rhs_vjp(up_d, cot_d, ns.Params(scatter="block"))
    assert ei.value.status == _abi.EUNSUPPORTED
    m.close()


def test_single_reference_tet_closed_form(dev):
    X = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], float)
    U = np.zeros((4, 4))
    U[1, 3] = 1.0
    coords, conn = X.T.copy(), np.arange(4, dtype=np.int32).reshape(4, 1)
    w = mg.Workload("ref", 1, coords, conn, U.T.copy(), 1.0, 1e-2)
    x, m = gpu_rhs(dev, w)
    exp = np.zeros((4, 4))
    exp[:, :3] = np.array([[-1, -1, -1], [1, 0, 0], [0, 1, 0], [0, 0, 1]]) / 24.0
    exp[0, 3], exp[1, 3] = 1 / (24 * 1e-2), -1 / (24 * 1e-2)
    assert np.abs(x.T - exp).max() < 1e-14
    m.close()


@pytest.mark.parametrize("tau", ["gauss", "element"])
def test_single_tet_vreman_feeds_tau_closed_form(dev, tau):
    """The 50-digit closed form with the Vreman model and every term on
    (mu_eff in the viscous term and in tau), through the C ABI, FP64 and
    mixed."""
    import test_oracle_pins as pins
    rho, mu, cv, s, q = 2.0, 1e-3, 0.1, 0.2, -1.3
    X, U = pins.vreman_stabilised_inputs(s, q)
    exp = pins.closed_form_vreman_stabilised(rho, mu, cv, s, q, tau == "element")
    coords, conn = X.T.copy(), np.arange(4, dtype=np.int32).reshape(4, 1)
    w = mg.Workload("ref", 1, coords, conn, U.T.copy(), rho, mu)
    for prec, tol in (("fp64", 1e-13), ("mixed", 1e-5)):
        x, m = gpu_rhs(dev, w, ns.Params(rho=rho, mu=mu, c_vreman=cv, tau=tau, precision=prec))
        assert np.abs(x.T - exp).max() <= tol * np.abs(exp).max(), prec
        m.close()


@pytest.mark.parametrize("n,cv", [(32, 0.0), (64, 0.0), (32, 0.07)])
def test_mixed_precision_error(dev, n, cv):
    w = mg.make_workload(n, jitter=0.3, order="rcm", mu=1e-4, mag_max=10.0, c_vreman=cv)
    ref = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu, c_vreman=cv)
    for scatter in ("auto", "atomic", "block"):
        x, m = gpu_rhs(dev, w, ns.Params(rho=w.rho, mu=w.mu, c_vreman=cv, precision="mixed",
                                         scatter=scatter))
        info = m.info()
        assert info["n_high_ar"] > 0            # the jitter-0.3 mesh has AR > 10 elements
        assert relerr(x, ref) <= TOL_MIXED, (scatter, relerr(x, ref))
        m.close()


@pytest.mark.parametrize("n,order,cv", [(8, "lex", 0.0), (8, "lex", 0.07), (20, "random", 0.0),
                                        (20, "rcm", 0.07)])
def test_vjp_matches_oracle(dev, n, order, cv):
    w = mg.make_workload(n, order=order, mu=1e-3, mag_max=2.0, c_vreman=cv)
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    ref = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu, c_vreman=cv)
    coords, conn, up, cot_d = on_dev(dev, w.coords, w.conn, w.up, cot)
    m = ns.Mesh(coords, conn)
    for scatter in ("auto", "atomic", "block"):
        g = m.assemble_vjp(up, cot_d, rho=w.rho, mu=w.mu, c_vreman=cv,
                           scatter=scatter).cpu().numpy()
        assert relerr(g, ref) <= TOL_VJP_ORACLE, (scatter, relerr(g, ref))
    m.close()


def test_vjp_central_differences_100_directions(dev):
    """<grad, d> against <w, (F(u + eps d) - F(u - eps d)) / 2 eps> for 100
    seeded directions on the 8^3 mesh, GPU forward in FP64, eps = 1e-6."""
    w = mg.tiny()
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    dirs = mg.normal((100, 4, w.n_nodes), seed=mg.SEED_DIRS)
    coords, conn, up, cot_d = on_dev(dev, w.coords, w.conn, w.up, cot)
    m = ns.Mesh(coords, conn)
    p = ns.Params(rho=w.rho, mu=w.mu)
    g = m.assemble_vjp(up, cot_d, p).cpu().numpy()
    eps = 1e-6
    worst = 0.0
    for d in dirs:
        dd = torch.from_numpy(d).to(dev)
        fp = m.assemble(up + eps * dd, p)
        fm = m.assemble(up - eps * dd, p)
        fd = float(torch.sum(cot_d * (fp - fm)).item()) / (2 * eps)
        ad = float(np.sum(g * d))
        worst = max(worst, abs(fd - ad) / max(abs(ad), 1e-30))
    assert worst <= TOL_VJP_FD, worst
    m.close()


def test_autograd_function(dev):
    w = mg.make_workload(6, order="random", c_vreman=0.07)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn)
    p = ns.Params(rho=w.rho, mu=w.mu, c_vreman=0.07)
    upg = up.clone().requires_grad_(True)
    rhs = ns.assemble(m, upg, p)
    cot = torch.from_numpy(mg.normal((4, w.n_nodes), seed=mg.SEED_COT)).to(dev)
    (g,) = torch.autograd.grad(rhs, upg, cot)
    g2 = m.assemble_vjp(up, cot, p)
    # same kernel; only the order of the atomic adds may differ between runs
    assert relerr(g.cpu().numpy(), g2.cpu().numpy()) <= 1e-14
    ref = oracle.vjp(w.coords, w.conn, w.up, cot.cpu().numpy(), w.rho, w.mu, c_vreman=0.07)
    assert relerr(g.cpu().numpy(), ref) <= TOL_VJP_ORACLE
    m.close()


def test_mesh_errors(dev):
    w = mg.make_workload(3)
    coords, conn = on_dev(dev, w.coords, w.conn)
    bad = conn.clone()
    bad[2, 5] = w.n_nodes  # out of range
    with pytest.raises(ns.NSRHSError) as ei:
        ns.Mesh(coords, bad)
    assert ei.value.status == _abi.EMESH
    bad = conn.clone()
    bad[2, 7] = -1
    with pytest.raises(ns.NSRHSError):
        ns.Mesh(coords, bad)
    inv = conn.clone()
    inv[[1, 2], 11] = inv[[2, 1], 11]  # swap two nodes: detJ < 0
    with pytest.raises(ns.NSRHSError) as ei:
        ns.Mesh(coords, inv)
    assert ei.value.status == _abi.EMESH
    m = ns.Mesh(coords, conn)
    up = torch.zeros((4, w.n_nodes), dtype=torch.float64, device=dev)
    with pytest.raises(TypeError):
        m.assemble(up.float())                    # wrong dtype for fp64
    with pytest.raises(ns.NSRHSError) as ei:
        m.assemble(up, ns.Params(mu=-1.0))        # invalid parameter
    assert ei.value.status == _abi.EINVAL
    with pytest.raises(TypeError):
        m.assemble_vjp(up, up, ns.Params(precision="mixed"))   # mixed takes float32
    m.close()
    with pytest.raises(RuntimeError):
        m.assemble(up)
    # the library kept working after the rejected calls
    x, m2 = gpu_rhs(dev, w)
    check_fp64(x, oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu))
    m2.close()


def test_constant_velocity_gives_zero(dev):
    w = mg.make_workload(10, order="random")
    up = np.zeros_like(w.up)
    up[:3] = np.array([0.3, -2.0, 1.1])[:, None]
    x, m = gpu_rhs(dev, w, ns.Params(rho=1.0, mu=1e-2, c_vreman=0.07), up=up)
    assert np.abs(x).max() < 1e-15
    m.close()


def test_step_pipeline_matches_direct_calls(dev):
    """The double-buffered host pipeline returns, step after step, what the
    direct calls return (same kernels; only atomic ordering may differ)."""
    w = mg.make_workload(12, order="rcm", mu=1e-3, mag_max=2.0)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn)
    p = ns.Params(rho=w.rho, mu=w.mu)
    ups = [w.up * s for s in (1.0, 0.5, -2.0, 3.0, 0.25)]
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    up_h = [torch.from_numpy(a).pin_memory() for a in ups]
    cot_h = torch.from_numpy(cot).pin_memory()
    rhs_h = [torch.empty((4, w.n_nodes), dtype=torch.float64).pin_memory() for _ in ups]
    grad_h = [torch.empty((4, w.n_nodes), dtype=torch.float64).pin_memory() for _ in ups]
    pipe = ns.StepPipeline(m, p)
    for k in range(len(ups)):
        pipe.submit(k, up_h[k], cot_h, rhs_h[k], grad_h[k])
    pipe.synchronize()
    cot_d = torch.from_numpy(cot).to(dev)
    for k, a in enumerate(ups):
        ad = torch.from_numpy(a).to(dev)
        r = m.assemble(ad, p).cpu().numpy()
        g = m.assemble_vjp(ad, cot_d, p).cpu().numpy()
        assert relerr(rhs_h[k].numpy(), r) <= 1e-14
        assert relerr(grad_h[k].numpy(), g) <= 1e-14
    # forward only (no cotangent), and the single-call host helper
    pipe = ns.StepPipeline(m, p)
    rhs2 = [torch.empty((4, w.n_nodes), dtype=torch.float64).pin_memory() for _ in ups]
    for k in range(len(ups)):
        pipe.submit(k, up_h[k], None, rhs2[k], None)
    pipe.synchronize()
    for k in range(len(ups)):
        assert relerr(rhs2[k].numpy(), rhs_h[k].numpy()) <= 1e-14
        assert relerr(ns.assemble_host(m, up_h[k], p).numpy(), rhs_h[k].numpy()) <= 1e-14
    m.close()


VARIANTS = [(cv, conv, tau) for cv in (0.0, 0.07) for conv in ("convective", "skew")
            for tau in ("gauss", "element")]


@pytest.mark.parametrize("cv,conv,tau", VARIANTS)
def test_formulation_variants_match_oracle(dev, cv, conv, tau):
    """Skew-symmetric convection and per-element tau (each with Vreman on and
    off): forward (FP64 atomic and block, mixed) and adjoint against the oracle."""
    w = mg.make_workload(14, jitter=0.2, order="random", mu=1e-3, mag_max=3.0, c_vreman=cv)
    okw = dict(c_vreman=cv, skew=conv == "skew", tau_elem=tau == "element")
    ref = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu, **okw)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn)
    for scatter in ("atomic", "block"):
        p = ns.Params(rho=w.rho, mu=w.mu, c_vreman=cv, convection=conv, tau=tau, scatter=scatter)
        check_fp64(m.assemble(up, p).cpu().numpy(), ref)
    pm = ns.Params(rho=w.rho, mu=w.mu, c_vreman=cv, convection=conv, tau=tau, precision="mixed")
    assert relerr(m.assemble(up.float(), pm).cpu().numpy(), ref) <= TOL_MIXED
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    gref = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu, **okw)
    for scatter in ("atomic", "block"):
        p = ns.Params(rho=w.rho, mu=w.mu, c_vreman=cv, convection=conv, tau=tau, scatter=scatter)
        g = m.assemble_vjp(up, torch.from_numpy(cot).to(dev), p).cpu().numpy()
        assert relerr(g, gref) <= TOL_VJP_ORACLE, (scatter, relerr(g, gref))
    m.close()


@pytest.mark.parametrize("cv,conv,tau", VARIANTS)
def test_recomputed_geometry_matches_oracle(dev, cv, conv, tau):
    """geometry='recompute' (Jacobian, cofactors, 1/detJ, detJ^(-1/3) formed
    from the gathered coordinates in the call): forward and adjoint against
    the oracle, every formulation variant, a ragged element count."""
    w = mg.make_workload(13, jitter=0.3, order="random", mu=1e-3, mag_max=3.0, c_vreman=cv)
    okw = dict(c_vreman=cv, skew=conv == "skew", tau_elem=tau == "element")
    ref = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu, **okw)
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    gref = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu, **okw)
    coords, conn, up, cot_d = on_dev(dev, w.coords, w.conn, w.up, cot)
    m = ns.Mesh(coords, conn)
    for scatter in ("auto", "atomic"):
        p = ns.Params(rho=w.rho, mu=w.mu, c_vreman=cv, convection=conv, tau=tau, scatter=scatter,
                      geometry="recompute")
        check_fp64(m.assemble(up, p).cpu().numpy(), ref)
        g = m.assemble_vjp(up, cot_d, p).cpu().numpy()
        assert relerr(g, gref) <= TOL_VJP_ORACLE, (scatter, relerr(g, gref))
    m.close()


def test_recomputed_geometry_unsupported_combinations(dev):
    w = mg.make_workload(4)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn, colour=True)
    for kw in (dict(scatter="block"), dict(scatter="colour"), dict(scatter="block_colour"),
               dict(precision="mixed")):
        p = ns.Params(geometry="recompute", **kw)
        u = up.float() if kw.get("precision") == "mixed" else up
        with pytest.raises(_abi.NSRHSError):
            m.assemble(u, p)
        with pytest.raises(_abi.NSRHSError):
            m.assemble_vjp(u, u, p)
    with pytest.raises(_abi.NSRHSError):
        m.assemble_rhs_vjp(up, up, ns.Params(geometry="recompute"))
    with pytest.raises(_abi.NSRHSError):
        m.assemble_elmat(up, ns.Params(geometry="recompute"))
    # out-of-range geometry and a nonzero reserved field are argument errors
    import ctypes
    lib = ns.load_library()
    out = torch.empty_like(up)
    for geo, res in ((2, 0), (-1, 0), (0, 1)):
        cp = ns.Params().to_c()
        cp.geometry, cp.reserved = geo, res
        st = lib.nsrhs_assemble(m.handle, ctypes.byref(cp), ctypes.c_void_p(up.data_ptr()),
                                ctypes.c_void_p(out.data_ptr()), None)
        assert st == _abi.EINVAL
    # the FP64 explicit step assembles through the recompute path
    w2 = up.clone()
    m.explicit_step(w2, 1e-4, "euler", ns.Params(geometry="recompute"))
    w3 = up.clone()
    m.explicit_step(w3, 1e-4, "euler", ns.Params())
    assert relerr(w2.cpu().numpy(), w3.cpu().numpy()) <= 1e-14
    m.close()


def test_skew_convection_does_no_work_on_gpu(dev):
    """The energy identity through the kernel: with the skew-symmetric form
    the convective RHS does no work, so with mu -> tiny, no pressure and no
    stabilisation-free shortcut, sum u . F over the convective part is zero.
    Checked as the difference of two assemblies that differ only in rho."""
    w = mg.make_workload(10, jitter=0.1, order="rcm", mag_max=1.0)
    up = w.up.copy()
    up[3] = 0.0
    coords, conn, upd = on_dev(dev, w.coords, w.conn, up)
    m = ns.Mesh(coords, conn)
    # the convective Galerkin term is the only one that is not stabilisation,
    # viscous, pressure or continuity: isolate it with the oracle's term mask
    ref_conv = oracle.assemble(w.coords, w.conn, up, 1.0, 1e-2, terms=oracle.T_CONV, skew=True)
    assert abs(np.sum(up[:3] * ref_conv[:3])) <= 1e-14 * np.sum(np.abs(up[:3] * ref_conv[:3]))
    full = m.assemble(upd, ns.Params(rho=1.0, mu=1e-2, convection="skew")).cpu().numpy()
    rest = oracle.assemble(w.coords, w.conn, up, 1.0, 1e-2,
                           terms=oracle.T_ALL & ~oracle.T_CONV, skew=True)
    conv_gpu = full - rest
    assert abs(np.sum(up[:3] * conv_gpu[:3])) <= 1e-12 * np.sum(np.abs(up[:3] * conv_gpu[:3]))
    m.close()


def test_lumped_mass_and_explicit_steps_match_oracle(dev):
    w = mg.make_workload(10, jitter=0.2, order="rcm", mu=1e-3, mag_max=2.0)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn)
    mass = m.lumped_mass().cpu().numpy()
    mref = oracle.lumped_mass(w.coords, w.conn)
    assert relerr(mass, mref) <= 1e-14
    dt = 2e-3
    for scheme in ("euler", "ssprk3"):
        for kw in ({}, {"convection": "skew", "c_vreman": 0.07}):
            u = up.clone()
            p = ns.Params(rho=w.rho, mu=w.mu, **{k: v for k, v in kw.items()})
            okw = {"skew": kw.get("convection") == "skew", "c_vreman": kw.get("c_vreman", 0.0)}
            ref = w.up.copy()
            for _ in range(3):
                m.explicit_step(u, dt, scheme, p)
                ref = oracle.explicit_step(w.coords, w.conn, ref, w.rho, w.mu, dt, scheme, **okw)
            got = u.cpu().numpy()
            # compare the change of the state (the increments carry the RHS)
            assert relerr(got - w.up, ref - w.up) <= 1e-12, (scheme, kw)
            assert np.array_equal(got[3], w.up[3])
    work = torch.empty((8, w.n_nodes), dtype=torch.float64, device=dev)
    with pytest.raises(ns.NSRHSError):
        m.explicit_step(up.clone(), -1.0, "euler", ns.Params(), work=work)
    with pytest.raises(ns.NSRHSError):
        m.explicit_step(up.clone(), 1e-3, "euler", ns.Params(rho=0.0), work=work)
    m.close()


@pytest.mark.parametrize("n,order", [(10, "rcm"), (16, "random")])
def test_unstructured_delaunay_mesh(dev, n, order):
    """Delaunay mesh of a jittered lattice (varying valence, no hex-block
    structure): FP64 atomic and block, mixed, adjoint, a variant, the mixed
    adjoint and the one-pass call (mixed, and FP64 on blocks)."""
    w = mg.make_unstructured(n, order=order, mu=1e-3, mag_max=2.0)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn)
    ref = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu)
    for scatter in ("atomic", "block"):
        check_fp64(m.assemble(up, ns.Params(rho=w.rho, mu=w.mu, scatter=scatter)).cpu().numpy(),
                   ref)
    x = m.assemble(up.float(), ns.Params(rho=w.rho, mu=w.mu, precision="mixed")).cpu().numpy()
    assert relerr(x, ref) <= TOL_MIXED
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    g = m.assemble_vjp(up, torch.from_numpy(cot).to(dev), rho=w.rho, mu=w.mu).cpu().numpy()
    assert relerr(g, oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu)) <= TOL_VJP_ORACLE
    sk = m.assemble(up, ns.Params(rho=w.rho, mu=w.mu, convection="skew")).cpu().numpy()
    check_fp64(sk, oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu, skew=True))
    # the mixed adjoint and the one-pass call on the block scatter (irregular
    # runs: node valences vary)
    gref = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu)
    pm = ns.Params(rho=w.rho, mu=w.mu, precision="mixed")
    cot32 = torch.from_numpy(cot).to(dev).float()
    assert relerr(m.assemble_vjp(up.float(), cot32, pm).cpu().numpy(), gref) <= TOL_VJP_FD
    r1, g1 = m.assemble_rhs_vjp(up.float(), cot32, pm)
    assert relerr(r1.cpu().numpy(), ref) <= TOL_MIXED
    assert relerr(g1.cpu().numpy(), gref) <= TOL_VJP_FD
    r2, g2 = m.assemble_rhs_vjp(up, torch.from_numpy(cot).to(dev),
                                ns.Params(rho=w.rho, mu=w.mu, scatter="block"))
    check_fp64(r2.cpu().numpy(), ref)
    assert relerr(g2.cpu().numpy(), gref) <= TOL_VJP_ORACLE
    m.close()


@pytest.mark.parametrize("cv", [0.0, 0.07])
def test_element_matrix_path_matches_oracle(dev, cv):
    """The element-matrix comparison path computes the same RHS."""
    w = mg.make_workload(12, jitter=0.2, order="random", mu=1e-3, mag_max=2.0, c_vreman=cv)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn)
    x = m.assemble_elmat(up, ns.Params(rho=w.rho, mu=w.mu, c_vreman=cv)).cpu().numpy()
    check_fp64(x, oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu, c_vreman=cv))
    with pytest.raises(ns.NSRHSError) as ei:
        m.assemble_elmat(up, ns.Params(convection="skew"))
    assert ei.value.status == _abi.EUNSUPPORTED
    m.close()


@pytest.mark.parametrize("cv,conv", [(0.0, "convective"), (0.07, "skew")])
def test_mixed_precision_adjoint(dev, cv, conv):
    """Float reverse sweep with double accumulation: within the adjoint's
    1e-6 tolerance against the oracle's complex-step element Jacobians."""
    w = mg.make_workload(20, jitter=0.3, order="rcm", mu=1e-3, mag_max=3.0, c_vreman=cv)
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    ref = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu, c_vreman=cv, skew=conv == "skew")
    coords, conn, up, cot_d = on_dev(dev, w.coords, w.conn, w.up, cot)
    m = ns.Mesh(coords, conn)
    for scatter in ("atomic", "block"):
        p = ns.Params(rho=w.rho, mu=w.mu, c_vreman=cv, convection=conv, precision="mixed",
                      scatter=scatter)
        g = m.assemble_vjp(up.float(), cot_d.float(), p).cpu().numpy()
        assert relerr(g, ref) <= TOL_VJP_FD, (scatter, relerr(g, ref))
    m.close()


@pytest.mark.parametrize("scatter", ["auto", "atomic", "block", "block_colour"])
@pytest.mark.parametrize("cv,conv,tau", [(0.0, "convective", "gauss"), (0.07, "convective", "gauss"),
                                         (0.0, "skew", "gauss"), (0.07, "skew", "element")])
def test_one_pass_rhs_and_vjp(dev, cv, conv, tau, scatter):
    """nsrhs_assemble_rhs_vjp: both outputs against the oracle (FP64 and
    mixed; auto is atomic for FP64 and blocks for mixed), on a mesh with a
    ragged element count."""
    w = mg.make_workload(11, jitter=0.2, order="random", mu=1e-3, mag_max=3.0, c_vreman=cv)
    okw = dict(c_vreman=cv, skew=conv == "skew", tau_elem=tau == "element")
    ref = oracle.assemble(w.coords, w.conn, w.up, w.rho, w.mu, **okw)
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    gref = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu, **okw)
    coords, conn, up, cot_d = on_dev(dev, w.coords, w.conn, w.up, cot)
    m = ns.Mesh(coords, conn, colour=scatter == "block_colour")
    kw = dict(rho=w.rho, mu=w.mu, c_vreman=cv, convection=conv, tau=tau, scatter=scatter)
    r, g = m.assemble_rhs_vjp(up, cot_d, ns.Params(**kw))
    check_fp64(r.cpu().numpy(), ref)
    assert relerr(g.cpu().numpy(), gref) <= TOL_VJP_ORACLE
    pm = ns.Params(precision="mixed", **kw)
    r, g = m.assemble_rhs_vjp(up.float(), cot_d.float(), pm)
    assert relerr(r.cpu().numpy(), ref) <= TOL_MIXED
    assert relerr(g.cpu().numpy(), gref) <= TOL_VJP_FD
    if scatter == "block_colour":   # fixed summation order: bitwise repeatable
        r2, g2 = m.assemble_rhs_vjp(up.float(), cot_d.float(), pm)
        assert torch.equal(r, r2) and torch.equal(g, g2)
    m.close()


def test_one_pass_blocks_match_separate_calls(dev):
    """The one-pass block kernel's two outputs against the separate block
    calls at the same state: the same staged gathers and per-node sums, the
    element RHS taken from the adjoint's recomputation, so they agree to
    rounding (FP64) and to the float element arithmetic (mixed)."""
    w = mg.make_workload(14, jitter=0.2, order="rcm", mu=1e-3, mag_max=2.0)
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    coords, conn, up, cot_d = on_dev(dev, w.coords, w.conn, w.up, cot)
    m = ns.Mesh(coords, conn)
    for prec, u, c, tol in (("fp64", up, cot_d, 1e-13), ("mixed", up.float(), cot_d.float(), 1e-6)):
        p = ns.Params(rho=w.rho, mu=w.mu, scatter="block", precision=prec)
        r, g = m.assemble_rhs_vjp(u, c, p)
        assert relerr(r.cpu().numpy(), m.assemble(u, p).cpu().numpy()) <= tol
        assert relerr(g.cpu().numpy(), m.assemble_vjp(u, c, p).cpu().numpy()) <= tol
    m.close()


def test_one_pass_argument_errors(dev):
    w = mg.make_workload(3)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn)
    out = torch.empty_like(up)
    with pytest.raises(ns.NSRHSError) as ei:
        m.assemble_rhs_vjp(up, up, ns.Params(), out=(out, out))
    assert ei.value.status == _abi.EINVAL
    with pytest.raises(ns.NSRHSError) as ei:
        m.assemble_rhs_vjp(up, up, ns.Params(scatter="colour"))
    assert ei.value.status == _abi.EUNSUPPORTED
    with pytest.raises(ns.NSRHSError) as ei:   # no block colouring on this mesh
        m.assemble_rhs_vjp(up, up, ns.Params(scatter="block_colour"))
    assert ei.value.status == _abi.EUNSUPPORTED
    m.close()


@pytest.mark.parametrize("scatter", ["auto", "colour"])
def test_step_graph_replays_the_direct_steps(dev, scatter):
    """Explicit steps captured in a CUDA graph give the direct calls' result
    (bitwise with the deterministic colour scatter)."""
    w = mg.make_workload(6, jitter=0.2, order="rcm", mu=1e-3, mag_max=2.0)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn, colour=scatter == "colour")
    p = ns.Params(rho=w.rho, mu=w.mu, scatter=scatter)
    direct = up.clone()
    for _ in range(3):
        m.explicit_step(direct, 2e-3, "ssprk3", p)
    graphed = up.clone()
    g = ns.StepGraph(m, graphed, 2e-3, "ssprk3", p, steps=3)
    assert torch.equal(graphed, up)          # capture does not advance the state
    g.replay()
    if scatter == "colour":
        assert torch.equal(graphed, direct)
    else:
        d = (graphed - up).cpu().numpy()
        ref = (direct - up).cpu().numpy()
        assert relerr(d, ref) <= 1e-13
    g.replay()                               # three more steps
    for _ in range(3):
        m.explicit_step(direct, 2e-3, "ssprk3", p)
    assert relerr((graphed - up).cpu().numpy(), (direct - up).cpu().numpy()) <= 1e-13
    m.close()


def test_mixed_explicit_steps_and_autograd(dev):
    """The mixed form inside the explicit step (float stage RHS, double state)
    and behind autograd (float32 up): both against the FP64 oracle within the
    mixed form's tolerances."""
    w = mg.make_workload(10, jitter=0.2, order="rcm", mu=1e-3, mag_max=2.0)
    coords, conn, up = on_dev(dev, w.coords, w.conn, w.up)
    m = ns.Mesh(coords, conn)
    pm = ns.Params(rho=w.rho, mu=w.mu, precision="mixed")
    for scheme in ("euler", "ssprk3"):
        u = up.clone()
        ref = w.up.copy()
        for _ in range(2):
            m.explicit_step(u, 2e-3, scheme, pm)
            ref = oracle.explicit_step(w.coords, w.conn, ref, w.rho, w.mu, 2e-3, scheme)
        assert u.dtype == torch.float64
        assert relerr(u.cpu().numpy() - w.up, ref - w.up) <= TOL_MIXED, scheme
    with pytest.raises(ValueError):   # the mixed step needs 10 rows of work
        m.explicit_step(up.clone(), 2e-3, "euler", pm,
                        work=torch.empty((8, w.n_nodes), dtype=torch.float64, device=dev))
    up32 = up.float().requires_grad_(True)
    rhs = ns.assemble(m, up32, pm)
    assert rhs.dtype == torch.float64
    assert relerr(rhs.detach().cpu().numpy(), oracle.assemble(w.coords, w.conn, w.up, w.rho,
                                                               w.mu)) <= TOL_MIXED
    cot = mg.normal((4, w.n_nodes), seed=mg.SEED_COT)
    (g,) = torch.autograd.grad(rhs, up32, torch.from_numpy(cot).to(dev))
    assert g.dtype == torch.float32
    gref = oracle.vjp(w.coords, w.conn, w.up, cot, w.rho, w.mu)
    assert relerr(g.double().cpu().numpy(), gref) <= TOL_VJP_FD
    m.close()


def test_adjoint_at_zero_velocity_matches_central_differences(dev):
    """At u = 0 every |u_g| is 0, where |u| has no derivative; the adjoint
    takes the symmetric (central-difference) value 0 for d|u_g|/du_g. Checked
    against central differences of the GPU forward on seeded directions."""
    # mu = 1 keeps c2 rho h / (c1 mu) small, so that tau varies little over
    # the difference step (tau(eps|d|) differs from tau(0) by O(eps))
    w = mg.make_workload(5, jitter=0.2, order="random", mu=1.0)
    up0 = w.up.copy()
    up0[:3] = 0.0
    coords, conn, up = on_dev(dev, w.coords, w.conn, up0)
    m = ns.Mesh(coords, conn)
    p = ns.Params(rho=1.0, mu=1.0)
    cot = torch.from_numpy(mg.normal((4, w.n_nodes), seed=mg.SEED_COT)).to(dev)
    g = m.assemble_vjp(up, cot, p).cpu().numpy()
    assert np.isfinite(g).all()
    dirs = mg.normal((10, 4, w.n_nodes), seed=mg.SEED_DIRS)
    eps = 1e-7
    for d in dirs:
        dd = torch.from_numpy(d).to(dev)
        fd = float(torch.sum(cot * (m.assemble(up + eps * dd, p) - m.assemble(up - eps * dd, p))))
        fd /= 2 * eps
        ad = float(np.sum(g * d))
        assert abs(fd - ad) <= TOL_VJP_FD * max(abs(ad), 1e-30), (fd, ad)
    m.close()


def test_calls_run_on_the_callers_stream(dev):
    """Every call is issued on the caller's current stream: inputs produced on
    a side stream, the calls issued there and only that stream synchronised
    give the default stream's results (no call synchronises the device or
    falls back to the default stream)."""
    w = mg.make_workload(10, jitter=0.2, order="rcm", mu=1e-3, mag_max=2.0)
    coords, conn, up, cot = on_dev(dev, w.coords, w.conn, w.up, mg.normal((4, w.n_nodes), seed=5))
    m = ns.Mesh(coords, conn, colour=True)
    p = ns.Params(rho=w.rho, mu=w.mu)
    ref = m.assemble(up, p).cpu().numpy()
    gref = m.assemble_vjp(up, cot, p).cpu().numpy()
    pm = ns.Params(rho=w.rho, mu=w.mu, precision="mixed")
    mref = m.assemble(up.float(), pm).cpu().numpy()
    torch.cuda.synchronize(dev)
    s = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(s):
        u2 = up * 1.0          # produced on the side stream
        c2 = cot * 1.0
        x = m.assemble(u2, p)
        g = m.assemble_vjp(u2, c2, p)
        r1, g1 = m.assemble_rhs_vjp(u2, c2, p)
        xm = m.assemble(u2.float(), pm)
        xc = m.assemble(u2, ns.Params(rho=w.rho, mu=w.mu, scatter="colour"))
    s.synchronize()
    for a, b in ((x, ref), (g, gref), (r1, ref), (g1, gref), (xc, ref)):
        assert relerr(a.cpu().numpy(), b) <= 1e-13
    assert relerr(xm.cpu().numpy(), mref) <= 1e-6
    m.close()
