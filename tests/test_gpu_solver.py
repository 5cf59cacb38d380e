"""GPU even/odd CG against the CPU oracle (through the C ABI).

The bar for every solve: the FP64 true residual
||phi - M x|| / ||phi||, recomputed by the ORACLE's operator on the GPU solution,
is below 1e-10.  On 4^4 the GPU solution is also compared with the oracle's own
even/odd solve.
"""
import numpy as np
import pytest

import oracle
from paper_0905_3331_gb300 import (CG_FP64, CG_RELIABLE, CG_SQRT_EPS, DF64, F16, F32, F64, LINK8,
                                   LINK12, LINK18, Lattice, TMError, inputs)

from _util import rel

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MODES = [
    ("fp64", dict(mode=CG_FP64)),
    ("sqrt_eps_f32_12", dict(mode=CG_SQRT_EPS, sloppy_prec=F32, sloppy_link=LINK12)),
    ("reliable_f32_18", dict(mode=CG_RELIABLE, sloppy_prec=F32, sloppy_link=LINK18)),
    ("reliable_f32_12", dict(mode=CG_RELIABLE, sloppy_prec=F32, sloppy_link=LINK12)),
    ("reliable_f16_12", dict(mode=CG_RELIABLE, sloppy_prec=F16, sloppy_link=LINK12)),
    ("reliable_f16_8", dict(mode=CG_RELIABLE, sloppy_prec=F16, sloppy_link=LINK8)),
    ("reliable_f32_12_df64_updates", dict(mode=CG_RELIABLE, sloppy_prec=F32, sloppy_link=LINK12,
                                          update_prec=DF64)),
]


def dev():
    return torch.device("cuda:0")


def oracle_true_residual(w, U, phi, x, f=1):
    olat = oracle.Lattice.cubic(w.T, w.L)
    r = phi - oracle.apply_M(olat, U, x, w.kappa, w.mu if f == 1 else -w.mu)
    return np.linalg.norm(r) / np.linalg.norm(phi)


@pytest.mark.parametrize("name,kw", MODES)
def test_solve_4x4x4x4(name, kw):
    w = inputs.WORKLOADS["4^4"]
    U, phi = w.gauge(), w.source()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(torch.from_numpy(U).to(dev()))
    b = torch.from_numpy(phi).to(dev())
    x = torch.zeros_like(b)
    info = lat.solve_cg(x, b, tol=1e-10, **kw)
    xn = x.cpu().numpy()
    assert oracle_true_residual(w, U, phi, xn) < 1e-10
    assert info.true_rel_residual < 1e-10 and info.schur_rel_residual < 1e-10
    # agreement with the oracle's own even/odd solve (both at 1e-12)
    lat.solve_cg(x, b, tol=1e-12, **kw)
    ref = oracle.solve(oracle.Lattice.cubic(w.T, w.L), U, phi, w.kappa, w.mu, tol=1e-12)
    assert rel(x.cpu().numpy(), ref.psi) < 1e-9
    lat.close()


@pytest.mark.parametrize("name,kw", [MODES[0], MODES[3], MODES[4], MODES[6]])
def test_solve_16x16x16x32(name, kw):
    """The 16^3 x 32 workload (eps 0.5, kappa 0.1632, mu 0.004), Gaussian source seed 2."""
    w = inputs.WORKLOADS["16^3x32"]
    U, phi = w.gauge(), w.source()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    b = torch.from_numpy(phi).to(dev())
    x = torch.zeros_like(b)
    info = lat.solve_cg(x, b, tol=1e-10, **kw)
    assert oracle_true_residual(w, U, phi, x.cpu().numpy()) < 1e-10
    assert info.iters > 0
    lat.close()


def test_flavour_minus_and_multiple_rhs():
    w = inputs.WORKLOADS["4^4"]
    U = w.gauge()
    phis = np.stack([w.source(k) for k in range(2)])
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    b = torch.from_numpy(phis).to(dev())
    x = torch.zeros_like(b)
    lat.solve_cg(x, b, nrhs=2, flavour=-1)
    xs = x.cpu().numpy()
    for k in range(2):
        assert oracle_true_residual(w, U, phis[k], xs[k], f=-1) < 1e-10
    # each system equals its own single solve
    x1 = torch.zeros_like(b[1])
    lat.solve_cg(x1, b[1].contiguous(), flavour=-1)
    assert torch.equal(x1, x[1])
    lat.close()


def test_deterministic_and_host_buffers():
    w = inputs.WORKLOADS["4^4"]
    U, phi = w.gauge(), w.source()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    b = torch.from_numpy(phi).to(dev())
    x1, x2 = torch.zeros_like(b), torch.zeros_like(b)
    i1 = lat.solve_cg(x1, b, mode=CG_RELIABLE, sloppy_prec=F16)
    i2 = lat.solve_cg(x2, b, mode=CG_RELIABLE, sloppy_prec=F16)
    assert torch.equal(x1, x2) and i1.iters == i2.iters
    xh = np.zeros_like(phi)
    i3 = lat.solve_cg(xh, phi, mode=CG_RELIABLE, sloppy_prec=F16)
    assert np.array_equal(xh, x1.cpu().numpy()) and i3.iters == i1.iters
    lat.close()


def test_initial_guess_defect_correction():
    w = inputs.WORKLOADS["4^4"]
    U, phi = w.gauge(), w.source()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    b = torch.from_numpy(phi).to(dev())
    x = torch.zeros_like(b)
    lat.solve_cg(x, b, tol=1e-4)
    info = lat.solve_cg(x, b, tol=1e-10, use_x0=True)
    assert oracle_true_residual(w, U, phi, x.cpu().numpy()) < 1e-10
    assert info.true_rel_residual < 1e-10
    lat.close()


def test_edge_cases():
    w = inputs.WORKLOADS["4^4"]
    U, phi = w.gauge(), w.source()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    b = torch.from_numpy(phi).to(dev())
    # zero source gives x = 0
    x = torch.ones_like(b)
    info = lat.solve_cg(x, torch.zeros_like(b))
    assert torch.count_nonzero(x) == 0 and info.iters == 0
    # max_iter reached: TM_ERR_NOT_CONVERGED, info filled, last iterate returned
    x = torch.zeros_like(b)
    info = lat.solve_cg(x, b, max_iter=5, check=False)
    assert info.status == 7 and info.iters >= 5 and info.schur_rel_residual > 1e-10
    assert torch.count_nonzero(x) > 0
    with pytest.raises(TMError) as e:
        lat.solve_cg(x, b, max_iter=5)
    assert e.value.status_name == "TM_ERR_NOT_CONVERGED"
    # non-finite source
    bad = b.clone()
    bad[0, 0, 0, 0, 0, 0] = float("nan")
    with pytest.raises(TMError) as e:
        lat.solve_cg(x, bad)
    assert e.value.status_name == "TM_ERR_NONFINITE"
    # bad parameters
    for kw in (dict(tol=0.0), dict(mode=7), dict(mode=CG_RELIABLE, delta=1.5),
               dict(flavour=3), dict(mode=CG_RELIABLE, sloppy_prec=0),
               dict(mode=CG_RELIABLE, update_prec=F16)):
        with pytest.raises(TMError) as e:
            lat.solve_cg(x, b, **kw)
        assert e.value.status_name == "TM_ERR_ARG"
    with pytest.raises(TMError):
        lat.solve_cg(b, b)
    lat.close()


def test_smallest_lattice_2x2x2x2():
    """2^4: the +mu and -mu neighbours of every site coincide."""
    U = inputs.random_gauge(2, 2, 0.6, 3)
    phi = inputs.gaussian_spinor(2, 2, 4)
    lat = Lattice(2, 2, 0.15, 0.05)
    lat.set_gauge(U)
    b = torch.from_numpy(phi).to(dev())
    for name, kw in MODES:
        x = torch.zeros_like(b)
        lat.solve_cg(x, b, **kw)
        olat = oracle.Lattice.cubic(2, 2)
        r = phi - oracle.apply_M(olat, U, x.cpu().numpy(), 0.15, 0.05)
        assert np.linalg.norm(r) / np.linalg.norm(phi) < 1e-10, name
    lat.close()


_SUBPROCESS_SOLVE = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_0905_3331_gb300 import Lattice, inputs, CG_RELIABLE, F16
w = inputs.WORKLOADS["4^4"]
lat = Lattice(w.T, w.L, w.kappa, w.mu)
for prec, link in ((0, 18), (2, 12)):
    lat.set_hop_threads(prec, link, 2)
lat.set_gauge(w.gauge())
b = torch.from_numpy(w.source()).cuda()
x = torch.zeros_like(b)
info = lat.solve_cg(x, b, mode=CG_RELIABLE, sloppy_prec=F16)
np.save({out!r}, x.cpu().numpy())
print("ITERS", info.iters)
"""


@pytest.mark.parametrize("env", [{"TM_NO_GRAPH": "1"}, {"TM_VERBOSE": "1"}, {"TM_PDL": "1"},
                                 {"TM_PDL": "1", "TM_NO_GRAPH": "1"}])
def test_host_loop_fallback_and_tracing(env, tmp_path):
    """The host-driven stage loop (TM_NO_GRAPH=1) and programmatic dependent launch (TM_PDL=1)
    give bitwise the same solution as the CUDA-graph loop (all reductions have a fixed order);
    TM_VERBOSE=1 traces the stages."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "x.npy")
    code = _SUBPROCESS_SOLVE.format(root=root, out=out)
    r = subprocess.run([sys.executable, "-c", code], env={**os.environ, **env}, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    w = inputs.WORKLOADS["4^4"]
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    for prec, link in ((0, 18), (2, 12)):  # same kernel choice as the subprocess
        lat.set_hop_threads(prec, link, 2)
    lat.set_gauge(w.gauge())
    b = torch.from_numpy(w.source()).to(dev())
    x = torch.zeros_like(b)
    info = lat.solve_cg(x, b, mode=CG_RELIABLE, sloppy_prec=F16)
    assert np.array_equal(np.load(out), x.cpu().numpy())
    assert f"ITERS {info.iters}" in r.stdout
    if "TM_VERBOSE" in env:
        assert "[tm_solve_cg] sloppy stage" in r.stderr and "reliable update" in r.stderr
    lat.close()


@pytest.mark.parametrize("tps", [1, 2, 4, 3, 5])
def test_solve_with_each_threads_per_site(tps):
    """Every launch configuration of the hopping kernel (3: the software-pipelined one, 5: two
    sites per thread with packed FP32 pairs, both for the FP32 / FP16 forms, FP64 then one thread
    per site) gives a solve that meets the bar."""
    w = inputs.WORKLOADS["4^4"]
    U, phi = w.gauge(), w.source()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    for prec, link in ((0, 18), (1, 12), (2, 12), (2, 8)):
        lat.set_hop_threads(prec, link, 1 if (tps in (3, 5) and prec == 0) else tps)
    lat.set_gauge(U)
    b = torch.from_numpy(phi).to(dev())
    for kw in (dict(mode=CG_FP64), dict(mode=CG_RELIABLE, sloppy_prec=F32, sloppy_link=LINK12),
               dict(mode=CG_RELIABLE, sloppy_prec=F16, sloppy_link=LINK12),
               dict(mode=CG_RELIABLE, sloppy_prec=F16, sloppy_link=LINK8, delta=0.3, update_prec=F32)):
        x = torch.zeros_like(b)
        lat.solve_cg(x, b, **kw)
        assert oracle_true_residual(w, U, phi, x.cpu().numpy()) < 1e-10
    assert lat.hop_threads(0, 18) == (1 if tps in (3, 5) else tps)
    assert lat.hop_threads(1, 12) == tps
    lat.close()


@pytest.mark.parametrize("name", ["16^3x32", "48^3x96"])
def test_paired_kernel_in_the_headline_solve(name):
    """The headline solve (FP16 storage, 8-real links, delta 0.3, FP32 recomputations between FP64
    ones) with the two-sites-per-thread hopping kernel: the oracle's residual of the GPU solution
    is below 1e-10."""
    w = inputs.WORKLOADS[name]
    U, phi = w.gauge(), w.source()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_hop_threads(F16, LINK8, 5)
    lat.set_hop_threads(F32, LINK8, 5)
    lat.set_gauge(U)
    b = torch.from_numpy(phi).to(dev())
    x = torch.zeros_like(b)
    info = lat.solve_cg(x, b, mode=CG_RELIABLE, sloppy_prec=F16, sloppy_link=LINK8, delta=0.3, update_prec=F32,
                        max_iter=20000)
    assert oracle_true_residual(w, U, phi, x.cpu().numpy()) < 1e-10 and info.true_rel_residual < 1e-10
    lat.close()


@pytest.mark.parametrize("name,sloppy,link,delta,upd", [
    ("32^3x64", F32, LINK12, 1e-3, F64),    # precision form: FP32 storage, 12-real links
    ("32^3x64", F16, LINK12, 0.1, F64),     # precision form: FP16 + norm storage, 12-real links
    ("32^3x64", F16, LINK12, 0.1, F32),     # the same with FP32 recomputations between FP64 ones
    ("48^3x96", F16, LINK8, 0.3, F64),      # large volume: FP16 storage, 8-real links (half)
    ("48^3x96", F16, LINK8, 0.3, F32),
])
def test_full_size_precision_forms(name, sloppy, link, delta, upd):
    """The 32^3 x 64 and 48^3 x 96 workloads solved to an FP64 true residual of 1e-10 with the
    reliable-update CG; the oracle recomputes the residual of the GPU solution on the host."""
    w = inputs.WORKLOADS[name]
    U, phi = w.gauge(), w.source()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    b = torch.from_numpy(phi).to(dev())
    x = torch.zeros_like(b)
    info = lat.solve_cg(x, b, mode=CG_RELIABLE, sloppy_prec=sloppy, sloppy_link=link, delta=delta,
                        max_iter=20000, update_prec=upd)
    res = oracle_true_residual(w, U, phi, x.cpu().numpy())
    assert res < 1e-10 and info.true_rel_residual < 1e-10
    assert abs(res - info.true_rel_residual) < 1e-3 * res
    lat.close()


def test_bench_configuration_16x16x16x32():
    """The solve bench.py times (16^3 x 32, FP32 storage, 12-real links, reliable updates at
    delta 1e-5, host and device buffers): the oracle's M applied to the GPU solution gives a true
    residual below 1e-10, and the reported residual agrees with it."""
    w = inputs.WORKLOADS["16^3x32"]
    U, phi = w.gauge(), w.source()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    b = torch.from_numpy(phi).to(dev())
    x = torch.zeros_like(b)
    kw = dict(mode=CG_RELIABLE, sloppy_prec=F32, sloppy_link=LINK12, delta=1e-5)
    info = lat.solve_cg(x, b, tol=1e-10, **kw)
    res = oracle_true_residual(w, U, phi, x.cpu().numpy())
    assert res < 1e-10 and abs(res - info.true_rel_residual) < 1e-3 * res
    xh = np.zeros_like(phi)
    lat.solve_cg(xh, phi, tol=1e-10, **kw)
    assert np.array_equal(xh, x.cpu().numpy())
    lat.close()


def test_multiple_rhs_reliable_mode_goes_through_the_batched_solver():
    """nrhs = 3 in the reliable-update mode: solved together (tm_solve_cg_batch inside
    tm_solve_cg); every solution meets the oracle-checked bar, device and host buffers alike."""
    w = inputs.WORKLOADS["8^4"]
    U = w.gauge()
    phis = np.stack([w.source(k) for k in range(3)])
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    kw = dict(mode=CG_RELIABLE, sloppy_prec=F32, sloppy_link=LINK12, delta=1e-3)
    b = torch.from_numpy(phis).to(dev())
    x = torch.zeros_like(b)
    info = lat.solve_cg(x, b, nrhs=3, flavour=-1, **kw)
    xs = x.cpu().numpy()
    for k in range(3):
        assert oracle_true_residual(w, U, phis[k], xs[k], f=-1) < 1e-10
    assert info.true_rel_residual < 1e-10
    xh = np.zeros_like(phis)
    lat.solve_cg(xh, phis, nrhs=3, flavour=-1, **kw)
    assert np.array_equal(xh, xs)
    lat.close()


_SUBPROCESS_DRIFT = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_0905_3331_gb300 import Lattice, inputs, CG_RELIABLE, F16, LINK8
w = inputs.WORKLOADS["8^4"]
lat = Lattice(w.T, w.L, w.kappa, w.mu)
lat.set_gauge(w.gauge())
b = torch.from_numpy(w.source()).cuda()
x = torch.zeros_like(b)
info = lat.solve_cg(x, b, mode=CG_RELIABLE, sloppy_prec=F16, sloppy_link=LINK8, delta=1e-12)
np.save({out!r}, x.cpu().numpy())
print("RES", info.true_rel_residual, info.schur_rel_residual, info.reliable_updates)
"""


def test_deferred_confirmation_falls_back(tmp_path):
    """In the mixed modes the last sloppy stage's convergence is confirmed by the FP64 residual of
    the full system.  With FP16 storage, 8-real links and no intermediate reliable update
    (delta 1e-12) the iterated residual drifts away from the true one, the confirmation fails,
    and the solve continues from X until the FP64 residual meets the bar (checked by the oracle)."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "x.npy")
    code = _SUBPROCESS_DRIFT.format(root=root, out=out)
    r = subprocess.run([sys.executable, "-c", code], env={**os.environ, "TM_VERBOSE": "1"}, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "not confirmed, continuing" in r.stderr
    assert "confirmation" in r.stderr and "(converged)" in r.stderr
    tr, sr, upd = r.stdout.split("RES")[1].split()
    assert float(tr) < 1e-10 and float(sr) < 1e-10 and int(upd) >= 2
    w = inputs.WORKLOADS["8^4"]
    assert oracle_true_residual(w, w.gauge(), w.source(), np.load(out)) < 1e-10


_SUBPROCESS_F32_UPDATES = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_0905_3331_gb300 import Lattice, inputs, CG_RELIABLE, F16, F32, LINK8, LINK12
w = inputs.WORKLOADS["12^3x24"]
lat = Lattice(w.T, w.L, w.kappa, w.mu)
lat.set_gauge(w.gauge())
b = torch.from_numpy(w.source()).cuda()
for k, link in enumerate((LINK12, LINK8)):
    x = torch.zeros_like(b)
    info = lat.solve_cg(x, b, mode=CG_RELIABLE, sloppy_prec=F16, sloppy_link=link, delta=0.1, update_prec=F32)
    np.save({out!r} + str(k) + ".npy", x.cpu().numpy())
    print("RES", info.true_rel_residual, info.reliable_updates)
"""


def test_fp32_recomputations_between_fp64_ones(tmp_path):
    """update_prec TM_F32 with FP16 storage: the reliable updates at delta are FP32 recomputations
    r = r64 - A dx relative to the last FP64 residual (traced), FP64 ones follow every factor
    1e-2, and the solutions meet the oracle-checked bar for 12- and 8-real links."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = str(tmp_path / "x")
    code = _SUBPROCESS_F32_UPDATES.format(root=root, out=out)
    r = subprocess.run([sys.executable, "-c", code], env={**os.environ, "TM_VERBOSE": "1"}, capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert "FP32 update" in r.stderr and "reliable update" in r.stderr
    w = inputs.WORKLOADS["12^3x24"]
    U, phi = w.gauge(), w.source()
    for k in range(2):
        assert oracle_true_residual(w, U, phi, np.load(out + str(k) + ".npy")) < 1e-10
    for line in r.stdout.split("RES")[1:]:
        assert float(line.split()[0]) < 1e-10


def test_update_prec_f32_in_every_mode():
    """TM_F32 recomputations are accepted by the sqrt(eps) mode and by tm_solve_normal too, and the
    results meet the bar."""
    w = inputs.WORKLOADS["8^4"]
    U, phi = w.gauge(), w.source()
    lat = Lattice(w.T, w.L, w.kappa, w.mu)
    lat.set_gauge(U)
    b = torch.from_numpy(phi).to(dev())
    x = torch.zeros_like(b)
    lat.solve_cg(x, b, mode=CG_SQRT_EPS, sloppy_prec=F16, sloppy_link=LINK12, delta=0.1, update_prec=F32)
    assert oracle_true_residual(w, U, phi, x.cpu().numpy()) < 1e-10
    lat.close()
