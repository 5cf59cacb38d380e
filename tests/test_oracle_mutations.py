"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in a copy of oracle/tm_oracle.c (a dropped term, a wrong sign,
a missing adjoint, a transposed operand, a misplaced boundary phase, a wrong inverse, a typo
in a gamma matrix ...), compiles it, swaps it in for the real oracle and runs the pins of
tests/test_oracle_pins.py at their smallest sizes: at least one pin must fail.  The CPU only.
"""
import os

import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "tm_oracle.c")

MUTATIONS = [
    ("projector sign swapped (1 - gamma) forward",
     "(s == t ? 1.0 : 0.0) + (double)dir * GAMMA[mu][s][t]",
     "(s == t ? 1.0 : 0.0) - (double)dir * GAMMA[mu][s][t]"),
    ("backward link not daggered",
     "link[a][b] = conj(u[3 * b + a]);", "link[a][b] = u[3 * a + b];"),
    ("backward link taken at x instead of x - mu",
     "const cplx *u = U + 36 * ln + 9 * mu;", "const cplx *u = U + 36 * lex + 9 * mu;"),
    ("forward link transposed",
     "for (int b = 0; b < 3; ++b) link[a][b] = u[3 * a + b];",
     "for (int b = 0; b < 3; ++b) link[a][b] = u[3 * b + a];"),
    ("antiperiodic phase dropped",
     "if (dir > 0 && c[mu] == g->n[mu] - 1) return unit_phase(theta[mu]);",
     "if (dir > 0 && c[mu] == g->n[mu] - 1) return 1.0;"),
    ("neighbour direction reversed",
     "cn[mu] = (c[mu] + dir + g->n[mu]) % g->n[mu];", "cn[mu] = (c[mu] - dir + g->n[mu]) % g->n[mu];"),
    ("twisted mass sign flipped",
     "cplx m = (s == t ? 1.0 : 0.0) + I * (double)f * mut * GAMMA[4][s][t];",
     "cplx m = (s == t ? 1.0 : 0.0) - I * (double)f * mut * GAMMA[4][s][t];"),
    ("twisted mass without gamma5",
     "cplx m = (s == t ? 1.0 : 0.0) + I * (double)f * mut * GAMMA[4][s][t];",
     "cplx m = (s == t ? 1.0 + I * (double)f * mut : 0.0);"),
    ("site-diagonal inverse with 1 - mu~^2",
     "out[12 * lex + k] = tmp[k] / (1.0 + mut * mut);", "out[12 * lex + k] = tmp[k] / (1.0 - mut * mut);"),
    ("kappa dropped from the hopping term of M",
     "out[12 * lex + 3 * s + a] = d[3 * s + a] - kappa * acc[s][a];",
     "out[12 * lex + 3 * s + a] = d[3 * s + a] - acc[s][a];"),
    ("Schur complement sign",
     "for (long k = 0; k < n; ++k) t4[k] -= t3[k];", "for (long k = 0; k < n; ++k) t4[k] += t3[k];"),
    ("source preparation sign",
     "varphi[i] = parity_of(c) == 0 ? ve[i] : phi[i] - t[i];",
     "varphi[i] = parity_of(c) == 0 ? ve[i] : phi[i] + t[i];"),
    ("reconstruction sign",
     "psi[12 * lex + k] = varphi[12 * lex + k] - u[12 * lex + k];",
     "psi[12 * lex + k] = varphi[12 * lex + k] + u[12 * lex + k];"),
    ("gamma_2 typo", "{{0, 0, 0, -1}, {0, 0, +1, 0}, {0, +1, 0, 0}, {-1, 0, 0, 0}},",
     "{{0, 0, 0, -1}, {0, 0, -1, 0}, {0, +1, 0, 0}, {-1, 0, 0, 0}},"),
    ("CG step length from <p, p>",
     "double alpha = rr / creal(dot(n, p, q));", "double alpha = rr / creal(dot(n, p, p));"),
    ("CG direction update without beta",
     "for (long i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];",
     "for (long i = 0; i < n; ++i) p[i] = r[i];"),
    ("BiCGstab omega conjugated", "cplx omega = tt > 0 ? dot(n, t, s) / tt : 0;",
     "cplx omega = tt > 0 ? dot(n, s, t) / tt : 0;"),
    ("BiCGstab beta without alpha / omega", "cplx beta = (rho_new / rho) * (alpha / omega);",
     "cplx beta = (rho_new / rho);"),
    ("BiCGstab direction update without omega v",
     "p[i] = r[i] + beta * (p[i] - omega * v[i]);", "p[i] = r[i] + beta * p[i];"),
    ("BiCGstab on Qhat instead of Mhat", "orc_schur(dims, theta, spread, kappa, mu, f, U, p, v, 0);",
     "orc_schur(dims, theta, spread, kappa, mu, f, U, p, v, 1);"),
    ("BiCGstab shadow residual not conjugated", "cplx rv = dot(n, rh, v);", "cplx rv = dot(n, v, rh);"),
    ("doublet splitting with tau3 instead of tau1", "eb * PAULI[1][f][f2] * (s == t ? 1.0 : 0.0);",
     "eb * PAULI[3][f][f2] * (s == t ? 1.0 : 0.0);"),
    ("doublet twisted mass without tau3", "I * mb * PAULI[3][f][f2] * GAMMA[4][s][t]",
     "I * mb * PAULI[0][f][f2] * GAMMA[4][s][t]"),
    ("doublet hopping on the other flavour", "v - kappa * hop[f * n + 12 * lex + 3 * s + a];",
     "v - kappa * hop[(1 - f) * n + 12 * lex + 3 * s + a];"),
    ("doublet adjoint without the flavour swap", "  gamma5_apply(g.V, in + n, t1);\n  gamma5_apply(g.V, in, t1 + n);",
     "  gamma5_apply(g.V, in, t1);\n  gamma5_apply(g.V, in + n, t1 + n);"),
    ("MR step length conjugated", "cplx alpha = dot(n, q, r) / qq;", "cplx alpha = dot(n, r, q) / qq;"),
    ("MR solution update along q", "for (long i = 0; i < n; ++i) x[i] += alpha * r[i];\n    for (long i = 0; i < n; ++i) r[i] -= alpha * q[i];\n    rr = norm2(n, r);\n    ++k;",
     "for (long i = 0; i < n; ++i) x[i] += alpha * q[i];\n    for (long i = 0; i < n; ++i) r[i] -= alpha * q[i];\n    rr = norm2(n, r);\n    ++k;"),
    ("tau2 typo", "{{0, -I}, {I, 0}},  /* tau^2  */", "{{0, I}, {-I, 0}},  /* tau^2  */"),
]

# the pins, at their smallest sizes
PIN_CALLS = [
    ("gamma", lambda: pins.test_gamma_matrices_clifford_algebra()),
    ("worked example", lambda: pins.test_point_source_worked_example()),
    ("free field M", lambda: pins.test_free_field_eigenvalues_of_M(2, 2)),
    ("free field MdagM", lambda: pins.test_free_field_spectrum_of_MdagM(4, 2, (0.0, 0.0, 0.0, 0.0))),
    ("gauge covariance", lambda: pins.test_gauge_covariance()),
    ("gamma5 hermiticity", lambda: pins.test_gamma5_hermiticity_with_twisted_mass()),
    ("boundary phases", lambda: pins.test_boundary_phase_placement_equivalence((1.0, 0.0, 0.0, 0.0))),
    ("diagonal inverse", lambda: pins.test_site_diagonal_inverse_is_the_inverse()),
    ("schur dense", lambda: pins.test_schur_operator_is_the_dense_schur_complement(2, 2)),
    ("solve dense", lambda: pins.test_even_odd_solve_equals_dense_solve(2, 2)),
    ("cg dense", lambda: pins.test_cg_on_normal_equations_matches_dense()),
    ("bicgstab = scipy", lambda: pins.test_bicgstab_iterates_match_scipy()),
    ("bicgstab dense", lambda: pins.test_bicgstab_solve_equals_dense_solve(2, 2)),
    ("mr identity", lambda: pins.test_mr_is_exact_in_one_step_for_the_identity()),
    ("mr monotone", lambda: pins.test_mr_residual_never_grows_and_solves_the_dense_system()),
    ("pauli", lambda: pins.test_pauli_matrices_algebra()),
    ("doublet eps 0", lambda: pins.test_doublet_without_splitting_is_two_twisted_flavours()),
    ("doublet free field", lambda: pins.test_doublet_free_field_spectrum()),
    ("doublet adjoint", lambda: pins.test_doublet_adjoint_relation()),
    ("doublet dense", lambda: pins.test_doublet_solve_equals_dense_solve(2, 2)),
]


# A planted mistake can make an iteration diverge: numpy's overflow warnings are expected there.
@pytest.mark.filterwarnings("ignore::RuntimeWarning")
@pytest.mark.parametrize("name,old,new", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_a_planted_mistake_fails_a_pin(name, old, new, tmp_path, monkeypatch):
    src = open(SRC).read()
    assert src.count(old) >= 1, f"mutation site not found: {old}"
    variant = oracle.load_library(oracle.compile_variant(src.replace(old, new, 1),
                                                         str(tmp_path / "libvariant.so")))
    monkeypatch.setattr(oracle, "_lib", variant)
    failed = []
    for pin, call in PIN_CALLS:
        try:
            call()
        except Exception:  # an assertion, a non-convergence, a numpy error: the pin caught it
            failed.append(pin)
    assert failed, f"no pin caught: {name}"


def test_the_unmutated_copy_passes_every_pin(tmp_path, monkeypatch):
    variant = oracle.load_library(oracle.compile_variant(open(SRC).read(), str(tmp_path / "libsame.so")))
    monkeypatch.setattr(oracle, "_lib", variant)
    for pin, call in PIN_CALLS:
        call()


# The chronological guess is plain numpy in oracle/__init__.py: its mistakes are planted in a
# copy of that function's source, and the chronological-guess pins must catch each.
CHRONO_MUTATIONS = [
    ("Galerkin matrix transposed", "G[j, i] = np.vdot(chis[j], Achi[i])", "G[i, j] = np.vdot(chis[j], Achi[i])"),
    ("right-hand side conjugated", "np.vdot(chis[j], phi)", "np.vdot(phi, chis[j])"),
    ("operator of the other flavour", "normal_op(lat, U, chi, kappa, mu, f)", "normal_op(lat, U, chi, kappa, mu, -f)"),
    ("coefficients conjugated in the guess", "X0 += c[i] * chis[i]", "X0 += np.conj(c[i]) * chis[i]"),
]

CHRONO_PINS = [
    ("exact on span", lambda: pins.test_chrono_guess_is_exact_on_its_span()),
    ("krylov = cg", lambda: pins.test_chrono_guess_with_a_krylov_history_is_the_cg_iterate()),
    ("minimises", lambda: pins.test_chrono_guess_minimises_the_error_functional()),
]


@pytest.mark.parametrize("name,old,new", CHRONO_MUTATIONS, ids=[m[0] for m in CHRONO_MUTATIONS])
def test_a_planted_mistake_in_the_chrono_guess_fails_a_pin(name, old, new, monkeypatch):
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(oracle.chrono_guess))
    assert src.count(old) == 1, f"mutation site not found: {old}"
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), "<mutated chrono_guess>", "exec"), ns)
    monkeypatch.setattr(oracle, "chrono_guess", ns["chrono_guess"])
    failed = []
    for pin, call in CHRONO_PINS:
        try:
            call()
        except Exception:
            failed.append(pin)
    assert failed, f"no pin caught: {name}"


# The correlator trace is plain numpy in oracle/__init__.py too: a transposed or conjugated
# Gamma, or the Gram matrix used transposed, must each fail the free-field correlator pin with
# Gamma != 1 (a mistake that Gamma = 1 would never show).
CORRELATOR_MUTATIONS = [
    ("Gamma transposed", "big = np.kron(np.asarray(G, dtype=np.complex128), np.eye(3))",
     "big = np.kron(np.asarray(G, dtype=np.complex128).T, np.eye(3))"),
    ("Gamma conjugated", "big = np.kron(np.asarray(G, dtype=np.complex128), np.eye(3))",
     "big = np.kron(np.conj(np.asarray(G, dtype=np.complex128)), np.eye(3))"),
    ("Gram matrix transposed", "np.trace(A[t] @ big)", "np.trace(A[t].T @ big)"),
]


@pytest.mark.parametrize("name,old,new", CORRELATOR_MUTATIONS, ids=[m[0] for m in CORRELATOR_MUTATIONS])
def test_a_planted_mistake_in_the_correlator_fails_its_pin(name, old, new, monkeypatch):
    import inspect
    import textwrap
    src = textwrap.dedent(inspect.getsource(oracle.correlator))
    assert src.count(old) == 1, f"mutation site not found: {old}"
    ns = dict(vars(oracle))
    exec(compile(src.replace(old, new), "<mutated correlator>", "exec"), ns)
    monkeypatch.setattr(oracle, "correlator", ns["correlator"])
    with pytest.raises(AssertionError):
        pins.test_free_field_correlators_with_gamma_from_momentum_space()
