"""The mixed solvers' deferred confirmation, forced to miss, for every solver that has one.

In the mixed modes a sloppy stage that reaches the tolerance is confirmed by the FP64 residual
of the full system that the reconstruction computes (its odd part is the Schur or normal-equation
residual up to the rounding of x_e).  If that residual misses the tolerance, the solve goes on
from the current solution with an FP64 recomputation, reusing the buffers the reconstruction
wrote.  Storage of low precision with no intermediate reliable update (delta 1e-12) lets the
iterated residual drift below the tolerance while the true one does not, so the confirmation
misses.  Each test runs the solve in a child process with TM_VERBOSE=1, checks the trace
("not confirmed, continuing" before a final "converged"; for the batched solve, whose FP64
service runs inside its single graph launch and checks the Schur residual ||b' - A X|| there,
the count of unconfirmed sloppy convergences in its per-system summary) and checks the solution with the
ORACLE's operator: ||b - M x|| / ||b|| < 1e-10.  (tm_solve_cg's own case is in
test_gpu_solver.py.)
"""
import os
import re
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_0905_3331_gb300 import inputs

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_PRELUDE = r"""
import sys, numpy as np, torch
sys.path.insert(0, {root!r})
from paper_0905_3331_gb300 import (Lattice, inputs, solve_cg_batch, CG_RELIABLE, F16, F32, LINK8)
w = inputs.WORKLOADS["8^4"]
"""


def run_child(body: str, tmp_path, tag: str):
    out = str(tmp_path / f"{tag}.npy")
    code = _PRELUDE.format(root=ROOT) + body.format(out=out)
    r = subprocess.run([sys.executable, "-c", code], env={**os.environ, "TM_VERBOSE": "1"},
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-4000:]
    return np.load(out), r.stderr


def assert_fell_back_then_converged(trace: str, name: str):
    lines = [ln for ln in trace.splitlines() if ln.startswith(f"[{name}]") and "confirmation" in ln]
    missed = [k for k, ln in enumerate(lines) if "not confirmed, continuing" in ln]
    done = [k for k, ln in enumerate(lines) if ln.endswith("(converged)")]
    assert missed, f"{name}: the confirmation never missed:\n" + "\n".join(lines)
    assert done and done[-1] > missed[0], f"{name}: no confirmed convergence after a miss:\n" + "\n".join(lines)


def oracle_rel(w, U, phi, x, kappa, mu):
    olat = oracle.Lattice.cubic(w.T, w.L)
    r = phi - oracle.apply_M(olat, U, x, kappa, mu)
    return np.linalg.norm(r) / np.linalg.norm(phi)


def test_doublet_confirmation_falls_back(tmp_path):
    body = r"""
lat = Lattice(w.T, w.L, w.kappa, w.mu)
lat.set_gauge(w.gauge())
b = torch.from_numpy(np.stack([w.source(0), w.source(1)])).cuda()
x = torch.zeros_like(b)
lat.solve_doublet(x, b, 0.15, 0.19, mode=CG_RELIABLE, sloppy_link=LINK8, delta=1e-12)
np.save({out!r}, x.cpu().numpy())
"""
    x, trace = run_child(body, tmp_path, "doublet")
    assert_fell_back_then_converged(trace, "tm_solve_doublet")
    w = inputs.WORKLOADS["8^4"]
    U = w.gauge()
    phi = np.stack([w.source(0), w.source(1)])
    olat = oracle.Lattice.cubic(w.T, w.L)
    r = phi - oracle.apply_Mh(olat, U, x, w.kappa, 0.15, 0.19)
    assert np.linalg.norm(r) / np.linalg.norm(phi) < 1e-10


def test_batch_confirmation_falls_back(tmp_path):
    body = r"""
lat = Lattice(w.T, w.L, w.kappa, w.mu)
lat.set_gauge(w.gauge())
bs = [torch.from_numpy(w.source(k)).cuda() for k in range(2)]
xs = [torch.zeros_like(b) for b in bs]
infos = solve_cg_batch([(lat, w.mu, xs[k], bs[k]) for k in range(2)], sloppy_prec=F16, sloppy_link=LINK8,
                       delta=1e-12)
np.save({out!r}, torch.stack(xs).cpu().numpy())
"""
    x, trace = run_child(body, tmp_path, "batch")
    # the batched solve confirms inside its graph: one summary line per system
    lines = [ln for ln in trace.splitlines() if ln.startswith("[tm_solve_cg_batch] system")]
    assert len(lines) == 2, trace[-4000:]
    missed = [int(re.search(r"(\d+) sloppy convergences not confirmed", ln).group(1)) for ln in lines]
    assert max(missed) >= 1, "the confirmation never missed:\n" + "\n".join(lines)
    assert all(", converged (" in ln for ln in lines), "\n".join(lines)
    assert all("one graph launch for the batch: yes" in ln for ln in lines), "\n".join(lines)
    w = inputs.WORKLOADS["8^4"]
    U = w.gauge()
    for k in range(2):
        assert oracle_rel(w, U, w.source(k), x[k], w.kappa, w.mu) < 1e-10


@pytest.mark.parametrize("solver,prec", [("bicgstab", "F16"), ("mr", "F32")])
def test_schur_solver_confirmation_falls_back(tmp_path, solver, prec):
    """BiCGstab and MR on Mhat (kappa 0.13, where the spectrum of Mhat lies in Re > 0)."""
    body = r"""
lat = Lattice(w.T, w.L, 0.13, w.mu)
lat.set_gauge(w.gauge())
b = torch.from_numpy(w.source()).cuda()
x = torch.zeros_like(b)
kw = dict(mode=CG_RELIABLE, sloppy_link=LINK8, delta=1e-12)
if {solver!r} == "bicgstab":
    lat.solve_bicgstab(x, b, sloppy_prec={prec}, **kw)
else:
    lat.solve_mr(x, b, **kw)
np.save({{out!r}}, x.cpu().numpy())
""".format(solver=solver, prec=prec)
    x, trace = run_child(body, tmp_path, solver)
    assert_fell_back_then_converged(trace, f"tm_solve_{solver}")
    w = inputs.WORKLOADS["8^4"]
    assert oracle_rel(w, w.gauge(), w.source(), x, 0.13, w.mu) < 1e-10
