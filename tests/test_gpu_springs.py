"""Spring-mass system on the edge relation (the paper's Figure 1 example)
against the FP64 oracle: positions, velocities and kinetic energy after a
few steps in both precisions, odd and even step counts, massless vertices,
bitwise reproducibility, and the calls' refusals."""
import numpy as np
import pytest
import torch

import meshgen
from oracle import springs
from _problems import rel_err

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def _abi():
    from paper_1506_07577_gb300 import abi
    return abi


def _case(n=3, seed=71, massless=()):
    m = meshgen.cube_grid(n, jitter=0.05, seed=seed)
    rng = np.random.default_rng(seed)
    q0 = m.X + 0.03 / n * rng.normal(size=m.X.shape)
    qd0 = 0.2 * rng.normal(size=m.X.shape)
    mass = rng.uniform(0.5, 2.0, size=m.n_verts)
    for v in massless:
        mass[v] = 0.0
    return m, q0, qd0, mass


def _oracle(m, q0, qd0, mass, k, dt, steps):
    e = springs.tet_edges(m.tets)
    rest = springs.rest_lengths(m.X, e)
    q, qd = springs.run(q0, qd0, mass, e, rest, k, dt, steps)
    return q, qd, springs.kinetic_energy(qd, mass)


def _gpu(m, q0, qd0, mass, k, dt, steps, prec, repeat=1):
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    dt_ = torch.float64 if prec == "f64" else torch.float32
    outs = []
    with DeviceTetMesh(m.X, m.tets, edges=True) as dm:
        dm.vertex_field("pos", dt_, value=m.X)
        abi.ebb_springs_init(dm.ctx, dm.tets, "pos")
        for _ in range(repeat):
            q = dm.vertex_field("q", dt_, value=q0)
            qd = dm.vertex_field("qd", dt_, value=qd0)
            dm.vertex_field("mass", dt_, ncomp=1, value=mass)
            e = abi.ebb_springs_run(dm.ctx, dm.tets, "q", "qd", "mass", k, dt, steps, energy=True)
            outs.append((q.double().cpu().numpy().T.copy(), qd.double().cpu().numpy().T.copy(), e))
    return outs


@pytest.mark.parametrize("prec", ["f64", "f32"])
@pytest.mark.parametrize("steps", [0, 1, 6])
def test_springs_match_oracle(prec, steps):
    m, q0, qd0, mass = _case()
    k, dt = 3.0, 2e-3
    qo, qdo, eo = _oracle(m, q0, qd0, mass, k, dt, steps)
    ((qg, qdg, eg),) = _gpu(m, q0, qd0, mass, k, dt, steps, prec)
    assert rel_err(qg, qo) < TOL[prec]
    assert rel_err(qdg, qdo) < TOL[prec]
    assert abs(eg - eo) <= TOL[prec] * 10 * eo


def test_massless_vertices_stay_and_runs_repeat_bitwise():
    m, q0, qd0, mass = _case(seed=72, massless=(0, 5))
    k, dt = 2.0, 1e-3
    qo, qdo, _ = _oracle(m, q0, qd0, mass, k, dt, 5)
    runs = _gpu(m, q0, qd0, mass, k, dt, 5, "f64", repeat=2)
    (qa, qda, ea), (qb, qdb, eb) = runs
    assert np.array_equal(qa, qb) and np.array_equal(qda, qdb) and ea == eb
    assert rel_err(qa, qo) < 1e-12
    for v in (0, 5):
        assert np.allclose(qa[v], q0[v] + 5 * dt * qd0[v], rtol=0, atol=1e-14)   # moves at constant velocity
        assert np.array_equal(qda[v], qd0[v])


def test_springs_refusals():
    abi = _abi()
    from paper_1506_07577_gb300.device_mesh import DeviceTetMesh
    m, q0, qd0, mass = _case(n=2, seed=73)
    with DeviceTetMesh(m.X, m.tets) as dm:                      # no edge relation
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_springs_init(dm.ctx, dm.tets, "X")
        assert ei.value.status == abi.EBB_ERR_STATE
    with DeviceTetMesh(m.X, m.tets, edges=True) as dm:
        dm.vertex_field("q", torch.float64, value=q0)
        dm.vertex_field("qd", torch.float64, value=qd0)
        dm.vertex_field("mass", torch.float64, ncomp=1, value=mass)
        dm.vertex_field("m32", torch.float32, ncomp=1, value=mass)
        with pytest.raises(abi.EbbError) as ei:                 # before init
            abi.ebb_springs_run(dm.ctx, dm.tets, "q", "qd", "mass", 1.0, 1e-3, 1)
        assert ei.value.status == abi.EBB_ERR_STATE
        abi.ebb_springs_init(dm.ctx, dm.tets, "X")
        with pytest.raises(abi.EbbError) as ei:                 # mixed dtypes
            abi.ebb_springs_run(dm.ctx, dm.tets, "q", "qd", "m32", 1.0, 1e-3, 1)
        assert ei.value.status == abi.EBB_ERR_ARG
        with pytest.raises(abi.EbbError) as ei:                 # same field twice
            abi.ebb_springs_run(dm.ctx, dm.tets, "q", "q", "mass", 1.0, 1e-3, 1)
        assert ei.value.status == abi.EBB_ERR_PHASE
        with pytest.raises(abi.EbbError) as ei:
            abi.ebb_springs_run(dm.ctx, dm.tets, "q", "qd", "mass", 1.0, 1e-3, -1)
        assert ei.value.status == abi.EBB_ERR_ARG
