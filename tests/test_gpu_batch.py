"""GPU batched solves (tm_solve_cg_batch) against the CPU oracle.

Every system of a batch must reach the same bar as a single solve: the oracle's own M
applied to the GPU solution gives ||phi - M x|| / ||phi|| < 1e-10.
"""
import numpy as np
import pytest

import oracle
from paper_0905_3331_gb300 import F16, F32, LINK12, LINK18, Lattice, TMError, inputs, solve_cg_batch

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def dev():
    return torch.device("cuda:0")


def oracle_rel_residual(T, L, U, phi, x, kappa, mu, f=1):
    olat = oracle.Lattice.cubic(T, L)
    r = phi - oracle.apply_M(olat, U, x, kappa, mu if f == 1 else -mu)
    return np.linalg.norm(r) / np.linalg.norm(phi)


@pytest.mark.parametrize("sloppy", [(F32, LINK12), (F16, LINK12), (F32, LINK18)])
def test_mixed_batch_of_lattices_masses_and_sources(sloppy):
    """Two lattices (4^4 and 4^3 x 6... as 6 x 4^3) with different gauge fields, three twisted
    masses and several sources, in one batched solve."""
    specs = [(4, 4, 0.3, 0.160, 11), (6, 4, 0.5, 0.1632, 12)]
    lats, gauges = [], []
    for T, L, eps, kappa, seed in specs:
        U = inputs.random_gauge(T, L, eps, seed)
        lat = Lattice(T, L, kappa, 0.01)
        lat.set_gauge(U)
        lats.append(lat)
        gauges.append(U)
    systems, meta = [], []
    for li, (T, L, eps, kappa, seed) in enumerate(specs):
        for mu in (0.002, 0.005, 0.01):
            for src in range(2):
                phi = inputs.gaussian_spinor(T, L, 100 + 10 * li + src)
                b = torch.from_numpy(phi).to(dev())
                x = torch.zeros_like(b)
                f = 1 if src == 0 else -1
                systems.append((lats[li], mu, x, b, f))
                meta.append((li, mu, phi, f))
    infos = solve_cg_batch(systems, sloppy_prec=sloppy[0], sloppy_link=sloppy[1], delta=0.1)
    for (lat, mu, x, b, f), (li, mu_, phi, f_), info in zip(systems, meta, infos):
        T, L, eps, kappa, seed = specs[li]
        res = oracle_rel_residual(T, L, gauges[li], phi, x.cpu().numpy(), kappa, mu, f)
        assert res < 1e-10, (li, mu, f, res)
        assert info.status == 0 and info.true_rel_residual < 1e-10 and info.iters > 0
    # the batched solution equals the single solve to within the solver tolerance
    lat, mu, x, b, f = systems[3]
    lat.set_params(lat.kappa, mu)
    x1 = torch.zeros_like(b)
    lat.solve_cg(x1, b, mode=2, sloppy_prec=sloppy[0], sloppy_link=sloppy[1], flavour=f, tol=1e-10)
    assert float(torch.linalg.vector_norm(x1 - x) / torch.linalg.vector_norm(x1)) < 1e-7
    for lat in lats:
        lat.close()


def test_twelve_point_sources_8x8x8x8():
    """The 12 spin-colour point sources of a propagator on one 8^4 lattice."""
    w = inputs.WORKLOADS["8^4"]
    U = w.gauge()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    systems, phis = [], []
    for s in range(4):
        for c in range(3):
            phi = inputs.point_source(w.T, w.L, s, c)
            b = torch.from_numpy(phi).to(dev())
            systems.append((lat, w.mu, torch.zeros_like(b), b))
            phis.append(phi)
    infos = solve_cg_batch(systems, sloppy_prec=F32, sloppy_link=LINK12, delta=1e-3)
    for (l, mu, x, b), phi, info in zip(systems, phis, infos):
        assert oracle_rel_residual(w.T, w.L, U, phi, x.cpu().numpy(), w.kappa, w.mu) < 1e-10
        assert info.true_rel_residual < 1e-10
    lat.close()


@pytest.mark.parametrize("sloppy,delta", [((F32, LINK12), 1e-3), ((F16, LINK12), 0.1)])
def test_batched_workload_at_full_size(sloppy, delta):
    """The batched workload at full size in ONE batched solve: the 12 spin-colour point sources on
    24^3 x 48 (eps 0.6, kappa 0.1615, mu 0.003) and the 8^4, 12^3 x 24 and 16^3 x 32 lattices
    (eps 0.5, kappa 0.1632) with 4 Gaussian sources for each mu in {0.002, 0.005, 0.01} -- 48
    systems on 4 gauge fields.  Every solution is checked with the ORACLE's M on the full lattice:
    ||phi - M x|| / ||phi|| < 1e-10."""
    defs = inputs.batched_workload()
    lats, gauges = {}, {}
    for d in defs:
        w = d.workload
        if w.name not in lats:
            gauges[w.name] = w.gauge()
            lats[w.name] = Lattice(w.T, w.L, w.kappa, w.mu)
            lats[w.name].set_gauge(gauges[w.name])
    systems = []
    for d in defs:
        b = torch.from_numpy(d.source()).to(dev())
        systems.append((lats[d.workload.name], d.mu, torch.zeros_like(b), b))
    infos = solve_cg_batch(systems, sloppy_prec=sloppy[0], sloppy_link=sloppy[1], delta=delta)
    for d, (lat, mu, x, b), info in zip(defs, systems, infos):
        w = d.workload
        res = oracle_rel_residual(w.T, w.L, gauges[w.name], d.source(), x.cpu().numpy(), w.kappa, d.mu)
        assert res < 1e-10, (w.name, d.mu, d.kind, d.index, res)
        assert info.status == 0 and info.true_rel_residual < 1e-10
    for lat in lats.values():
        lat.close()


def test_batch_edge_cases():
    w = inputs.WORKLOADS["4^4"]
    U = w.gauge()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    phi = w.source()
    b = torch.from_numpy(phi).to(dev())
    zero = torch.zeros_like(b)
    x0, x1 = torch.ones_like(b), torch.zeros_like(b)
    infos = solve_cg_batch([(lat, w.mu, x0, zero), (lat, w.mu, x1, b)])
    assert torch.count_nonzero(x0) == 0 and infos[0].iters == 0
    assert oracle_rel_residual(w.T, w.L, U, phi, x1.cpu().numpy(), w.kappa, w.mu) < 1e-10
    infos = solve_cg_batch([(lat, w.mu, x1, b)], max_iter=3, check=False)
    assert infos[0].status == 7
    with pytest.raises(TMError) as e:
        solve_cg_batch([(lat, w.mu, x1, b)], max_iter=3)
    assert e.value.status_name == "TM_ERR_NOT_CONVERGED"
    host = np.zeros_like(phi)
    with pytest.raises(TMError) as e:
        solve_cg_batch([(lat, w.mu, host, b)])
    assert e.value.status_name == "TM_ERR_ARG"
    lat.close()


_BATCH_CHILD = """
import numpy as np, torch
from paper_0905_3331_gb300 import Lattice, inputs, solve_cg_batch, F32, LINK12
w = inputs.WORKLOADS["4^4"]
lat = Lattice(w.T, w.L, w.kappa, w.mu)
for prec, link in ((0, 18), (1, 12)):  # fixed kernel choice: no timing-dependent tuning
    lat.set_hop_threads(prec, link, 1)
lat.set_gauge(w.gauge())
systems = []
for k, mu in enumerate((0.01, 0.02, 0.05)):
    b = torch.from_numpy(w.source(k)).cuda()
    systems.append((lat, mu, torch.zeros_like(b), b))
infos = solve_cg_batch(systems, sloppy_prec=F32, sloppy_link=LINK12, delta=0.01)
np.save({out!r}, torch.stack([s[2] for s in systems]).cpu().numpy())
print("ITERS", [i.iters for i in infos])
"""


@pytest.mark.parametrize("split", [("TM_BATCH_TPS", "1"), ("TM_BATCH_K", "2")])
def test_batch_host_loop_matches_graph_loop(tmp_path, split):
    """TM_NO_GRAPH=1 runs the batched loop (iteration, FP64 service) from the host: bitwise the same
    solutions, for a fixed batch split (the tuner's choice depends on timing)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for k, e in enumerate(({}, {"TM_NO_GRAPH": "1"})):
        out = str(tmp_path / f"x{k}.npy")
        r = subprocess.run([sys.executable, "-c", _BATCH_CHILD.format(out=out)], cwd=root,
                           env={**os.environ, **e, split[0]: split[1]}, capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stderr
        outs.append((np.load(out), r.stdout))
    assert np.array_equal(outs[0][0], outs[1][0]) and outs[0][1] == outs[1][1]


_SPLIT_CHILD = """
import sys, numpy as np, torch
from paper_0905_3331_gb300 import Lattice, inputs, solve_cg_batch, F16, F32, LINK8, LINK12
specs = [(4, 4, 0.3, 0.160, 11), (6, 4, 0.5, 0.1632, 12)]
lats = []
for T, L, eps, kappa, seed in specs:
    lat = Lattice(T, L, kappa, 0.01)
    lat.set_gauge(inputs.random_gauge(T, L, eps, seed))
    lats.append(lat)
systems = []
for li, (T, L, eps, kappa, seed) in enumerate(specs):
    for k, mu in enumerate((0.002, 0.005, 0.01, 0.02, 0.05)):  # 5 systems a lattice: a ragged last group
        b = torch.from_numpy(inputs.gaussian_spinor(T, L, 200 + 10 * li + k)).cuda()
        systems.append((lats[li], mu, torch.zeros_like(b), b, 1 if k % 2 == 0 else -1))
for prec, link in ((F32, LINK12), (F16, LINK8)):
    for s in systems:
        s[2].zero_()
    infos = solve_cg_batch(systems, sloppy_prec=prec, sloppy_link=link, delta=0.1)
    np.savez({out!r}.replace(".npy", "_%d_%d.npz" % (prec, link)), *[s[2].cpu().numpy() for s in systems])
    print("ITERS", prec, link, [i.iters for i in infos])
"""


@pytest.mark.parametrize("split", [("TM_BATCH_K", "2"), ("TM_BATCH_K", "4"), ("TM_BATCH_TPS", "2"),
                                   ("TM_BATCH_TPS", "4")])
def test_every_batch_split_solves_to_the_oracle(tmp_path, split):
    """Each batch split the tuner can pick -- K = 2 or 4 systems per thread (groups of one lattice,
    a ragged last group), or one system per thread with 2 or 4 threads per site -- forced through
    the environment, on two lattices with five systems each (both flavours), FP32/12 and FP16/8:
    every solution meets the oracle's residual bar."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "x.npy")
    r = subprocess.run([sys.executable, "-c", _SPLIT_CHILD.format(out=out)], cwd=root,
                       env={**os.environ, split[0]: split[1], "TM_VERBOSE": "1"}, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-4000:]
    specs = [(4, 4, 0.3, 0.160, 11), (6, 4, 0.5, 0.1632, 12)]
    for prec, link in ((F32, LINK12), (F16, 8)):
        z = np.load(out.replace(".npy", "_%d_%d.npz" % (prec, link)))
        xs = [z["arr_%d" % i] for i in range(len(z.files))]
        n = 0
        for li, (T, L, eps, kappa, seed) in enumerate(specs):
            U = inputs.random_gauge(T, L, eps, seed)
            for k, mu in enumerate((0.002, 0.005, 0.01, 0.02, 0.05)):
                phi = inputs.gaussian_spinor(T, L, 200 + 10 * li + k)
                f = 1 if k % 2 == 0 else -1
                res = oracle_rel_residual(T, L, U, phi, xs[n], kappa, mu, f)
                assert res < 1e-10, (split, prec, link, li, mu, res)
                n += 1


def test_batch_of_forty_systems_on_one_lattice():
    """40 systems on one lattice: the work lists compact their candidates 32 at a time (two
    ballots on this lattice), and with 4 systems per thread the ten groups fill one list too.
    Every solution meets the oracle's bar."""
    import os
    w = inputs.WORKLOADS["4^4"]
    U = w.gauge()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    systems, phis = [], []
    for k in range(40):
        phi = inputs.gaussian_spinor(w.T, w.L, 500 + k)
        b = torch.from_numpy(phi).to(dev())
        systems.append((lat, 0.005 + 0.001 * (k % 7), torch.zeros_like(b), b, 1 if k % 3 else -1))
        phis.append(phi)
    for split in (None, "4"):
        if split:
            os.environ["TM_BATCH_K"] = split
        try:
            for s in systems:
                s[2].zero_()
            infos = solve_cg_batch(systems, sloppy_prec=F32, sloppy_link=LINK12, delta=0.1)
        finally:
            os.environ.pop("TM_BATCH_K", None)
        for (lat_, mu, x, b, f), phi, info in zip(systems, phis, infos):
            res = oracle_rel_residual(w.T, w.L, U, phi, x.cpu().numpy(), w.kappa, mu, f)
            assert res < 1e-10 and info.status == 0, (split, mu, f, res)
    lat.close()
