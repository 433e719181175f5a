"""GPU parity of the implicit backward-Euler step (Jacobi PCG) against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import meshgen
from oracle import fem, implicit
from _problems import rel_err

pytestmark = pytest.mark.gpu

G = (0.0, 0.0, -9.81)


def _abi():
    from paper_1506_07577_gb300 import abi
    return abi


def _setup(n, model, per_tet, seed, jitter=0.01):
    m = meshgen.cube_grid(n, jitter=jitter, seed=seed)
    if per_tet:
        mu, lam = meshgen.material_loguniform_E(m.n_tets, 1e4, 1e6, 0.4, seed)
    else:
        mu, lam = (float(a) for a in meshgen.lame_from_young(1e5, 0.45))
    return m, mu, lam


def _oracle_steps(m, mu, lam, model, steps, dt, rho, max_iters, rtol, u0=None, v0=None):
    B, V = fem.rest_shape(m.X, m.tets)
    mass = fem.lumped_mass(V, m.tets, rho, m.n_verts)
    u = np.zeros_like(m.X) if u0 is None else u0.copy()
    v = np.zeros_like(m.X) if v0 is None else v0.copy()
    infos = []
    for _ in range(steps):
        u, v, info = implicit.implicit_step(m.X, u, v, m.tets, B, V, mass, mu, lam,
                                            fem.STVK if model == "stvk" else fem.NEOHOOKEAN,
                                            dt, np.array(G), m.pinned, max_iters, rtol)
        infos.append(info)
    return u, v, infos


def _gpu_steps(m, mu, lam, model, steps, dt, rho, max_iters, rtol, precision, reduce="tiled",
               pin_dtype=torch.uint8, u0=None, v0=None, fail_on_max=False):
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    per_tet = np.ndim(mu) > 0
    with DeviceTetMesh(m.X, m.tets, mu if per_tet else None, lam if per_tet else None,
                       colour=(reduce == "colour")) as dm:
        dm.vertex_field("u", torch.float64, value=np.zeros_like(m.X) if u0 is None else u0)
        dm.vertex_field("v", torch.float64, value=np.zeros_like(m.X) if v0 is None else v0)
        dm.bind("pinned", torch.from_numpy(m.pinned.astype(np.uint8)).to(dm.device, pin_dtype))
        prm = abi.step_params(abi.EBB_STVK if model == "stvk" else abi.EBB_NEOHOOKEAN, dt, rho,
                              0.0 if per_tet else mu, 0.0 if per_tet else lam, G,
                              abi.EBB_PREC_F64 if precision == "f64" else abi.EBB_PREC_F32,
                              {"atomic": abi.EBB_REDUCE_ATOMIC, "colour": abi.EBB_REDUCE_COLOR,
                               "tiled": abi.EBB_REDUCE_TILED, "gather": abi.EBB_REDUCE_GATHER,
                               "ordered": abi.EBB_REDUCE_TILED_ORDERED, "coop": abi.EBB_REDUCE_COOP}[reduce],
                              max_iters, rtol, fail_on_max)
        reps = []
        for _ in range(steps):
            reps.append(abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", "pinned", prm))
        u = dm._tensors["u"].cpu().numpy().T.copy()
        v = dm._tensors["v"].cpu().numpy().T.copy()
    return u, v, reps


@pytest.mark.parametrize("reduce", ["atomic", "colour", "tiled", "gather", "ordered", "coop"])
def test_stvk_fp64_step_n8_matches_oracle(reduce):
    """8x8x8 StVK FP64 workload: one step, dt = 1e-3, 50 CG iterations
    (early stop at 1e-14 relative residual)."""
    m, mu, lam = _setup(8, "stvk", False, seed=1)
    uo, vo, io = _oracle_steps(m, mu, lam, "stvk", 1, 1e-3, 1000.0, 50, 1e-14)
    ug, vg, rg = _gpu_steps(m, mu, lam, "stvk", 1, 1e-3, 1000.0, 50, 1e-14, "f64", reduce)
    assert abs(rg[0].iters - io[0]["iters"]) <= 1
    assert rel_err(vg, vo) < 1e-12
    assert rel_err(ug, uo) < 1e-12


@pytest.mark.parametrize("model", ["stvk", "nh"])
def test_fp64_multistep_matches_oracle(model):
    m, mu, lam = _setup(5, model, True, seed=4)
    v0 = 0.05 * meshgen.random_field(m.n_verts, seed=2)
    v0[m.pinned] = 0
    # CG run to 1e-14 on both sides, so that the solver's stopping error stays
    # below the FP64 parity bound of 1e-12
    uo, vo, io = _oracle_steps(m, mu, lam, model, 3, 2e-3, 1000.0, 400, 1e-14, v0=v0)
    ug, vg, rg = _gpu_steps(m, mu, lam, model, 3, 2e-3, 1000.0, 400, 1e-14, "f64", v0=v0)
    assert rel_err(vg, vo) < 1e-12
    assert rel_err(ug, uo) < 1e-12
    assert all(abs(a.iters - b["iters"]) <= 2 for a, b in zip(rg, io))


@pytest.mark.parametrize("pin_dtype,reduce", [(torch.uint8, "tiled"), (torch.int32, "tiled"),
                                              (torch.uint8, "gather"), (torch.uint8, "ordered"),
                                              (torch.uint8, "coop")])
def test_mixed_nh_steps_match_oracle(pin_dtype, reduce):
    """Mixed precision (FP32 element maps, FP64 CG) neo-Hookean with E
    log-uniform in [1e4, 1e6]: error against the FP64 oracle after 4 steps
    at rtol 1e-8."""
    m, mu, lam = _setup(8, "nh", True, seed=2)
    uo, vo, _ = _oracle_steps(m, mu, lam, "nh", 4, 1e-3, 1000.0, 1000, 1e-8)
    ug, vg, rg = _gpu_steps(m, mu, lam, "nh", 4, 1e-3, 1000.0, 1000, 1e-8, "f32", reduce=reduce,
                            pin_dtype=pin_dtype)
    assert all(r.rel_residual <= 1e-8 for r in rg)
    assert rel_err(vg, vo) < 1e-5
    assert rel_err(ug, uo) < 1e-5


@pytest.mark.parametrize("reduce", ["colour", "gather", "ordered"])
def test_atomic_free_step_is_bitwise_deterministic(reduce):
    m, mu, lam = _setup(6, "nh", True, seed=9)
    a = _gpu_steps(m, mu, lam, "nh", 2, 1e-3, 1000.0, 200, 1e-10, "f32", reduce)
    b = _gpu_steps(m, mu, lam, "nh", 2, 1e-3, 1000.0, 200, 1e-10, "f32", reduce)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_step_edge_cases():
    abi = _abi()
    m, mu, lam = _setup(3, "stvk", False, seed=3)
    # zero iterations allowed: dv = 0, v unchanged, u += dt v
    v0 = 0.1 * meshgen.random_field(m.n_verts, seed=1)
    ug, vg, rg = _gpu_steps(m, mu, lam, "stvk", 1, 1e-3, 1000.0, 0, 1e-8, "f64", v0=v0)
    assert rg[0].iters == 0
    assert np.array_equal(vg, v0) and np.allclose(ug, 1e-3 * v0, rtol=0, atol=1e-18)
    # hitting the cap above tolerance reports NOT_CONVERGED when asked
    with pytest.raises(abi.EbbError) as ei:
        _gpu_steps(m, mu, lam, "stvk", 1, 1e-3, 1000.0, 1, 1e-14, "f64", fail_on_max=True)
    assert ei.value.status == abi.EBB_ERR_NOT_CONVERGED
    # the cap is exact: iteration counts match the oracle's
    uo, vo, io = _oracle_steps(m, mu, lam, "stvk", 1, 1e-3, 1000.0, 3, 1e-14)
    ug, vg, rg = _gpu_steps(m, mu, lam, "stvk", 1, 1e-3, 1000.0, 3, 1e-14, "f64")
    assert rg[0].iters == io[0]["iters"] == 3
    assert rel_err(vg, vo) < 1e-12


def test_negative_density_rejected_on_host():
    """rho <= 0 is an argument error caught before any launch."""
    abi = _abi()
    m, mu, lam = _setup(2, "stvk", False, seed=3)
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    with DeviceTetMesh(m.X, m.tets) as dm:
        dm.vertex_field("u", torch.float64)
        dm.vertex_field("v", torch.float64)
        prm = abi.step_params(abi.EBB_STVK, 1e-3, 1000.0, mu, lam, G, max_iters=50, rtol=1e-12)
        prm.rho = -1000.0
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", None, prm)
        assert ei.value.status == abi.EBB_ERR_ARG   # rejected on the host: rho must be > 0


def test_breakdown_detected_on_device():
    """Negative Lame parameters make A = M + dt^2 K indefinite: the device
    detects p^T A p <= 0 and the step returns EBB_ERR_CG_BREAKDOWN."""
    abi = _abi()
    m, _, _ = _setup(2, "stvk", False, seed=3)
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    with DeviceTetMesh(m.X, m.tets) as dm:
        dm.vertex_field("u", torch.float64)
        dm.vertex_field("v", torch.float64)
        prm = abi.step_params(abi.EBB_STVK, 0.1, 1000.0, -1e8, -1e8, G, max_iters=50, rtol=1e-12)
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_cg_implicit_step(dm.ctx, dm.tets, "u", "v", None, prm)
        assert ei.value.status == abi.EBB_ERR_CG_BREAKDOWN


@pytest.mark.parametrize("prec", ["f32", "f64"])
def test_full_size_step_residual_sampled(prec):
    """At the benchmark size (64^3, neo-Hookean, E log-uniform, from a moving
    deformed state) the step's linear system is checked at sampled free
    vertices: the oracle forms b_i and (A dv)_i exactly from the tets around
    vertex i (A = M + dt^2 K(x_n), b = dt (f + M g - dt K v)), with dv the
    GPU's velocity change; the residual there is bounded by the solve's
    tolerance (|r_i| <= ||r||_2 <= rtol ||b||_2), and u' = u + dt v'."""
    from _problems import submesh_for_vertices
    n, dt, rho, rtol = 64, 1e-3, 1000.0, 1e-8
    m, mu, lam = _setup(n, "nh", True, seed=2)
    u0 = meshgen.random_displacement(m.X, n, amp=0.02, seed=7, smooth=0.01)
    v0 = 0.05 * meshgen.random_field(m.n_verts, seed=8)
    v0[m.pinned] = 0.0
    ug, vg, rg = _gpu_steps(m, mu, lam, "nh", 1, dt, rho, 1000, rtol, prec, u0=u0, v0=v0)
    assert rg[0].rel_residual <= rtol
    free = np.flatnonzero(~m.pinned)
    sample = np.random.default_rng(0).choice(free, size=64, replace=False)
    sel = np.isin(m.tets, sample).any(axis=1)
    sub = m.tets[sel]
    B, V = fem.rest_shape(m.X, sub)
    x = m.X + u0
    dv = vg - v0
    mdl = fem.NEOHOOKEAN
    f = fem.tet_forces(x, sub, B, V, mu[sel], lam[sel], mdl, m.n_verts)[sample]
    kv = fem.tet_Kv(x, v0, sub, B, V, mu[sel], lam[sel], mdl, m.n_verts)[sample]
    kdv = fem.tet_Kv(x, dv, sub, B, V, mu[sel], lam[sel], mdl, m.n_verts)[sample]
    mass = fem.lumped_mass(V, sub, rho, m.n_verts)[sample][:, None]
    b = dt * (f + mass * np.array(G) - dt * kv)
    Adv = mass * dv[sample] + dt * dt * kdv
    # ||b||_2 over all free rows from the oracle would need the whole mesh;
    # bound it by sqrt(3 N_free) times the sampled maximum's scale instead
    bound = rtol * np.sqrt(3 * free.size) * np.max(np.abs(b))
    assert np.max(np.abs(Adv - b)) <= 10 * bound
    assert np.max(np.abs(Adv - b)) <= 1e-4 * np.max(np.abs(b))
    np.testing.assert_allclose(ug[sample], u0[sample] + dt * vg[sample], rtol=0, atol=1e-15)
