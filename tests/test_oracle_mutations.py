"""Mutation checks of the oracle's pins.

Each case plants one plausible mistake in a copy of ``oracle/mdwf_oracle.c``
(a flipped sign, a dropped or doubled factor, the coefficient of the wrong row,
a transposed solve, a missing adjoint), builds that copy with gcc on the CPU,
loads it in place of the oracle's library and runs the pins named for the case:
at least one of them must fail. The committed oracle is never modified; the
mutated library is loaded for the duration of one case only. This shows that
the pins of ``test_oracle_pins.py``, ``test_oracle_sdep_pins.py``,
``test_oracle_chem_pins.py`` and ``test_oracle_force_ext_pins.py`` can tell
these mistakes apart from the paper's definitions.
"""
import contextlib
import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

import oracle
import synthetic as sy
import test_oracle_chem_pins as chem
import test_oracle_force_ext_pins as fext
import test_oracle_pins as base
import test_oracle_sdep_pins as sdep

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "mdwf_oracle.c")

TINY_DIMS = (4, 2, 2, 2)


def _tiny():
    return TINY_DIMS, sy.gauge_field(TINY_DIMS, 0.3, 11)


def _sdep_tiny():
    return TINY_DIMS, sy.gauge_field(TINY_DIMS, 0.3, 21)


# pins, each a callable taking the oracle module
PIN = {
    "gamma_basis": lambda o: base.test_gamma_basis(o),
    "free_wilson": lambda o: base.test_free_wilson_plane_waves(o),
    "lambda_max": lambda o: base.test_lambda_max_shamir(o),
    "dagger": lambda o: base.test_ddw_dagger_is_adjoint(o, _tiny(), 1.5, 0.5),
    "covariance": lambda o: base.test_gauge_covariance(o, _tiny()),
    "shamir": lambda o: base.test_shamir_limit_textbook(o, _tiny()),
    "blocks": lambda o: base.test_blocks_and_schur_complement(o, _tiny(), 1.5, 0.5),
    "solve": lambda o: base.test_solve_matches_dense_inverse(o, _tiny(), 1.5, 0.5),
    "force": lambda o: base.test_force_finite_differences(o),
    "adjoint_solve": lambda o: base.test_adjoint_solve_inverts_the_adjoint(o, _tiny()),
    "sdep_dagger": lambda o: sdep.test_dagger_is_adjoint(o, _sdep_tiny(), sdep.GENERIC),
    "sdep_overlap": lambda o: sdep.test_transfer_matrix_overlap_identity(o, _sdep_tiny(), sdep.GENERIC),
    "sdep_blocks": lambda o: sdep.test_blocks_schur_complement_and_solve(o, _sdep_tiny()),
    "chem_gamma5": lambda o: chem.test_gamma5_relation(o),
    "chem_free": lambda o: chem.test_free_field_shifted_momentum(o),
    "force_slices": lambda o: fext.test_per_slice_force_against_differences(o, 0.0),
    "force_chem": lambda o: fext.test_chemical_potential_force_against_differences(o),
}

# name -> (text in the oracle source, its replacement, pins of which one must fail)
MUTATIONS = {
    "gamma4_not_hermitian_unit": (
        "A[3][1][1] = 1;", "A[3][1][1] = -1;", ["gamma_basis", "free_wilson"]),
    "wilson_mass_plus_M5": (
        "out[12 * i + k] = (4.0 - M5) * in[12 * i + k] - 0.5 * h[k];",
        "out[12 * i + k] = (4.0 + M5) * in[12 * i + k] - 0.5 * h[k];", ["free_wilson", "lambda_max"]),
    "hopping_projectors_swapped": (
        "double sf = dagger ? +1.0 : -1.0;", "double sf = dagger ? -1.0 : +1.0;", ["free_wilson"]),
    "backward_link_not_adjoint": (
        "acc_spin_colour(out, wb, Sb, U + 9 * (4 * bw + mu), 1, fb);",
        "acc_spin_colour(out, wb, Sb, U + 9 * (4 * bw + mu), 0, fb);", ["dagger", "covariance"]),
    "chem_not_exchanged_in_adjoint": (
        "wf = exp(dagger ? -chem : chem);", "wf = exp(chem);", ["chem_free", "chem_gamma5"]),
    "wall_sign_flipped": (
        "double wp = (s == Ls - 1) ? -p->mf : 1.0;   /* coefficient of the s+1 block */",
        "double wp = (s == Ls - 1) ? p->mf : 1.0;   /* coefficient of the s+1 block */", ["shamir"]),
    "m_minus_sign": (
        "c.v[s] = c5_of(p, s) * (4.0 - p->M5) - 1.0;", "c.v[s] = c5_of(p, s) * (4.0 - p->M5) + 1.0;",
        ["blocks"]),
    "closed_form_power": (
        "acc += kappa * pow(-r, s) * b[(long)s * stride];",
        "acc += kappa * pow(-r, s + 1) * b[(long)s * stride];", ["blocks"]),
    "closed_form_transposed": (
        "solve_arr(xm + k, bm + k, n, Ls, Mp, Mm, p->mf, dagger ? 1 : 0);",
        "solve_arr(xm + k, bm + k, n, Ls, Mp, Mm, p->mf, dagger ? 0 : 1);", ["blocks"]),
    "per_slice_adjoint_takes_own_row": (
        "dw_affine(t, in + sp * n, U, p->L, p->M5, p->mu, 1, c5_of(p, sp), -1.0);",
        "dw_affine(t, in + sp * n, U, p->L, p->M5, p->mu, 1, c5_of(p, s), -1.0);", ["sdep_dagger"]),
    "per_slice_forward_takes_next_row": (
        "proj_field(t, PM, in + sp * n, V);\n            dw_affine(u, t, U, p->L, p->M5, p->mu, 0, c5_of(p, s), -1.0);",
        "proj_field(t, PM, in + sp * n, V);\n            dw_affine(u, t, U, p->L, p->M5, p->mu, 0, c5_of(p, sp), -1.0);",
        ["sdep_overlap", "sdep_blocks"]),
    "per_slice_ee_inverse_not_transposed": (
        "chiral_block(A, p, 1, dagger);", "chiral_block(A, p, 1, 0);", ["sdep_blocks"]),
    "prepare_drops_even_source": (
        "for (long k = 0; k < n; ++k) t[k] = bo[k] - u[k];", "for (long k = 0; k < n; ++k) t[k] = bo[k];",
        ["solve"]),
    "reconstruct_sign": (
        "for (long k = 0; k < n; ++k) t[k] = be[k] - t[k];", "for (long k = 0; k < n; ++k) t[k] = be[k] + t[k];",
        ["solve"]),
    "force_link_term_halved": (
        "acc_link_derivative(dSdU, a, w, p, 1, 2.0);", "acc_link_derivative(dSdU, a, w, p, 1, 1.0);", ["force"]),
    "force_dc5_keeps_d_plus_part": (
        "double dHd = which == 0 ? 1.0 : 0.0,", "double dHd = 1.0,", ["force"]),
    "force_time_factor_inverted": (
        "const double wf = (mu == 3 && p->mu != 0.0) ? exp(p->mu) : 1.0;",
        "const double wf = (mu == 3 && p->mu != 0.0) ? exp(-p->mu) : 1.0;", ["force_chem"]),
    "force_per_slice_rows_inverted": (
        "if (k != slice) cId.v[k]", "if (k == slice) cId.v[k]", ["force_slices"]),
    "force_action_from_wrong_vectors": (
        "*S = creal(dotc(phi, X, n));", "*S = creal(dotc(X, X, n));", ["force"]),
    "forward_link_at_neighbour": (
        "acc_spin_colour(out, wf, Sf, U + 9 * (4 * i + mu), 0, ff);",
        "acc_spin_colour(out, wf, Sf, U + 9 * (4 * fw + mu), 0, ff);", ["covariance", "dagger"]),
    "chem_on_a_space_direction": (
        "if (mu == 3 && chem != 0.0) {", "if (mu == 2 && chem != 0.0) {", ["chem_free"]),
    "cg_beta_inverted": (
        "double beta = rr_new / rr;\n            for (long i = 0; i < n; ++i) pp[i] = r[i] + beta * pp[i];\n"
        "            rr = rr_new;\n        }\n    }",
        "double beta = rr / rr_new;\n            for (long i = 0; i < n; ++i) pp[i] = r[i] + beta * pp[i];\n"
        "            rr = rr_new;\n        }\n    }", ["solve"]),
    "adjoint_solve_wrong_rhs": (
        "or_ddw(rhs, b, U, p, 0);", "or_ddw(rhs, b, U, p, 1);", ["adjoint_solve"]),
    "m_plus_sign": (
        "c.v[s] = b5_of(p, s) * (4.0 - p->M5) + 1.0;", "c.v[s] = b5_of(p, s) * (4.0 - p->M5) - 1.0;",
        ["blocks"]),
    "schur_complement_sign": (
        "for (long k = 0; k < n; ++k) out[k] = in[k] - b[k];", "for (long k = 0; k < n; ++k) out[k] = in[k] + b[k];",
        ["blocks"]),
    "m_dagger_inner_inverse_not_adjoint": (
        "or_mee_inv(a, b, Vh, p, 1);        /* I_rr^-dag (even) */",
        "or_mee_inv(a, b, Vh, p, 0);        /* I_rr^-dag (even) */", ["blocks"]),
    "cg_step_halved": (
        "            double alpha = rr / pap;\n            for (long i = 0; i < n; ++i) { x[i] += alpha * pp[i];",
        "            double alpha = 0.5 * rr / pap;\n            for (long i = 0; i < n; ++i) { x[i] += alpha * pp[i];",
        ["solve"]),
}


def _compile(out, text):
    src = out + ".c"
    with open(src, "w") as f:
        f.write(text)
    cmd = ["gcc", "-O2", "-std=c11", "-fcx-limited-range", "-fopenmp", "-fPIC", "-shared", "-o", out, src, "-lm"]
    subprocess.run(cmd, check=True, capture_output=True)
    return out


@pytest.fixture(scope="module")
def mutants(tmp_path_factory):
    """Builds every mutated copy once (in parallel); name -> shared-library path."""
    with open(SRC) as f:
        source = f.read()
    d = tmp_path_factory.mktemp("oracle_mutants")
    jobs = {}
    for name, (old, new, _) in MUTATIONS.items():
        assert source.count(old) == 1, f"{name}: the text to mutate must occur exactly once"
        jobs[name] = (str(d / f"lib_{name}.so"), source.replace(old, new))
    jobs["unmutated"] = (str(d / "lib_unmutated.so"), source)
    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {name: ex.submit(_compile, path, text) for name, (path, text) in jobs.items()}
        return {name: f.result() for name, f in futs.items()}


@contextlib.contextmanager
def _loaded(path):
    """The oracle module with its library replaced by the one at ``path``."""
    saved, real_build = oracle._lib, oracle.build
    oracle._lib = None
    oracle.build = lambda force=False: path
    try:
        oracle._load()
        yield oracle
    finally:
        oracle.build = real_build
        oracle._lib = saved


def test_pins_pass_on_an_unmutated_copy(oracle_lib, mutants):
    """The harness itself: the oracle's source built and loaded the same way as the
    mutants passes every pin, so a failure below comes from the planted mistake."""
    with _loaded(mutants["unmutated"]) as o:
        assert o._lib is not None
        for name, pin in PIN.items():
            pin(o)


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_mutation_fails_a_pin(oracle_lib, mutants, name):
    pins = MUTATIONS[name][2]
    caught = []
    with _loaded(mutants[name]) as o:
        for pin in pins:
            try:
                PIN[pin](o)
            except AssertionError:
                caught.append(pin)
    assert caught, f"mutation {name} passed every pin of {pins}"
