"""Planted mistakes: the oracle's pins must catch each of them.

Every mutant below is a copy of oracle/oracle.c with one plausible error in it: a dropped term
or factor, a wrong sign, a wrong index or operand, a wrong constant, a wrong tie or boundary
rule. Each copy is compiled on its own, loaded in place of the oracle (NAO_ORACLE_LIB), and the
oracle's pin tests (tests/test_oracle_*.py: closed forms, library routines, invariants, finite
differences, brute force) are run against it. A mutant survives if they all still pass; the test
fails if any mutant survives, or if the pin named beside it is not among those that fail. The
unmodified oracle passes the same pins in the rest of the suite.

The mutants are compiled under oracle/lib/mutants/ (a build folder, not tracked)."""
import os
import re
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor
from pathlib import Path

import pytest

ROOT = Path(__file__).resolve().parents[1]
SRC = ROOT / "oracle" / "oracle.c"
OUT = ROOT / "oracle" / "lib" / "mutants"
PINS = sorted(str(p.relative_to(ROOT)) for p in (ROOT / "tests").glob("test_oracle_*.py"))

# (name, text in oracle.c (must occur once), replacement, a pin test that must fail)
MUTANTS = [
    # radial splines (Sec. 3.2.1: cubic splines of the tabulated radial functions)
    ("spline system right-hand side halved",
     "double rhs = 6.0 * (", "double rhs = 3.0 * (",
     "test_spline_matches_scipy_natural_spline"),
    ("Thomas algorithm diagonal 4 -> 2",
     "double den = 4.0 - c[i - 1];", "double den = 2.0 - c[i - 1];",
     "test_spline_matches_scipy_natural_spline"),
    ("spline slope sign",
     "*dval = (y[k + 1] - y[k]) +", "*dval = (y[k] - y[k + 1]) +",
     "test_gradient_matches_finite_differences"),
    ("chain rule dr/ds loses 1/r",
     "    *R = v;\n    *dR = dv / (rr * delta);\n}", "    *R = v;\n    *dR = dv / delta;\n}",
     "test_gradient_matches_finite_differences"),
    ("cutoff not applied",
     "    if (r >= S->fn_cutoff[f]) { *R = 0.0; *dR = 0.0; return; }\n", "",
     "test_spline_interpolates_nodes_and_cutoff"),
    ("second radial derivative: sign of the dv term",
     "- dv / (rr * rr * delta);", "+ dv / (rr * rr * delta);",
     "test_radial_second_derivative"),
    # real spherical harmonics
    ("Legendre recurrence coefficient",
     "(double)(l + m - 1) * P[l - 2][m]", "(double)(l + m) * P[l - 2][m]",
     "test_ylm_orthonormal_to_l6"),
    ("Condon-Shortley phase added",
     "        P[m][m] = pmm;", "        P[m][m] = (m & 1) ? -pmm : pmm;",
     "test_ylm_textbook_low_orders"),
    ("normalisation 4 pi -> 2 pi",
     "double K = sqrt((2.0 * l + 1.0) / (4.0 * M_PI)", "double K = sqrt((2.0 * l + 1.0) / (2.0 * M_PI)",
     "test_ylm_orthonormal_to_l6"),
    ("cos and sin swapped between +m and -m",
     "Y[l + m] = M_SQRT2 * K * P[l][m] * c;\n            Y[l - m] = M_SQRT2 * K * P[l][m] * s;",
     "Y[l + m] = M_SQRT2 * K * P[l][m] * s;\n            Y[l - m] = M_SQRT2 * K * P[l][m] * c;",
     "test_ylm_textbook_low_orders"),
    ("dY/dtheta sign for m = 0",
     "if (m == 0) dP = -P[l][1];", "if (m == 0) dP = P[l][1];",
     "test_gradient_matches_finite_differences"),
    ("dY/dphi loses the factor m",
     "dYp_over_st[l + m] = -M_SQRT2 * K * Pm_over_st * (double)m * s;",
     "dYp_over_st[l + m] = -M_SQRT2 * K * Pm_over_st * s;",
     "test_gradient_matches_finite_differences"),
    ("theta unit vector: sign of its z component",
     "            double th[3] = {ct * cp, ct * sp_, -st};", "            double th[3] = {ct * cp, ct * sp_, st};",
     "test_gradient_matches_finite_differences"),
    ("Legendre P_{m+1}^m coefficient",
     "P[m + 1][m] = (double)(2 * m + 1) * x * pmm;", "P[m + 1][m] = (double)(2 * m - 1) * x * pmm;",
     "test_ylm_matches_scipy"),
    ("factorial ratio of the normalisation inverted",
     "factorial(l - m) / factorial(l + m));", "factorial(l + m) / factorial(l - m));",
     "test_ylm_orthonormal_to_l6"),
    ("angular part of the gradient loses 1/r",
     "grad[3 * cnt + c] = dR * Y[m] * rh[c] + (R / r) * (dYt[m]", "grad[3 * cnt + c] = dR * Y[m] * rh[c] + R * (dYt[m]",
     "test_gradient_matches_finite_differences"),
    # solid harmonics and the Cartesian second derivatives
    ("solid harmonic coefficient sign",
     "((sgn_exp & 1) ? -1.0 : 1.0)", "((sgn_exp & 1) ? 1.0 : -1.0)",
     "test_solid_harmonics_match_ylm_and_are_harmonic"),
    ("solid harmonic y exponent",
     "P->e[P->n][1] = 2 * u + w;", "P->e[P->n][1] = 2 * u;",
     "test_solid_harmonics_match_ylm_and_are_harmonic"),
    ("solid harmonic normalisation of m = 0",
     "(m == 0 ? 2.0 : 1.0)", "(m == 0 ? 1.0 : 2.0)",
     "test_solid_harmonics_match_ylm_and_are_harmonic"),
    ("monomial second derivative e(e - 1) -> e^2",
     "(double)(e[c] * (e[c] - 1))", "(double)(e[c] * e[c])",
     "test_solid_harmonic_derivatives_match_differences"),
    ("basis Hessian loses a cross term",
     "(g1 / r) * (x[ib] * Sg[ia] + x[ia] * Sg[ib])", "(g1 / r) * (x[ib] * Sg[ia])",
     "test_basis_hessian_laplacian_and_differences"),
    ("g'' coefficient 2l -> l",
     "- 2.0 * (double)l * dR / (rl * r)", "- (double)l * dR / (rl * r)",
     "test_basis_hessian_laplacian_and_differences"),
    # Hamiltonian (Eq. H_int_aims with the symmetric kinetic form)
    ("kinetic factor 1/2 dropped",
     "double tk = kin ? wp * 0.5 * gg : 0.0;\n                double tt", "double tk = kin ? wp * gg : 0.0;\n                double tt",
     "test_single_atom_closed_forms"),
    ("potential v dropped",
     "double tv = pot ? wp * (phi[a] * vp * phi[b]) : 0.0;", "double tv = pot ? wp * (phi[a] * phi[b]) : 0.0;",
     "test_single_atom_closed_forms"),
    ("z term of grad phi_i . grad phi_j dropped",
     "double gg = grad[3 * a] * grad[3 * b] + grad[3 * a + 1] * grad[3 * b + 1] + grad[3 * a + 2] * grad[3 * b + 2];",
     "double gg = grad[3 * a] * grad[3 * b] + grad[3 * a + 1] * grad[3 * b + 1];",
     "test_single_atom_closed_forms"),
    ("H element added to the wrong column",
     "size_t e = row + (size_t)idx[b];\n                neu_add(&H[e]", "size_t e = row + (size_t)idx[a];\n                neu_add(&H[e]",
     "test_two_centre_gaussian_product"),
    ("block Hamiltonian: kinetic factor 1/2 dropped",
     "double tk = kin ? wp * 0.5 * gg : 0.0;\n                size_t e = (size_t)a * (size_t)nF",
     "double tk = kin ? wp * gg : 0.0;\n                size_t e = (size_t)a * (size_t)nF",
     "test_block_equals_full"),
    ("brute force: kinetic factor 1/2 dropped",
     "0.5 * (gi[3 * i] * gi[3 * j]", "1.0 * (gi[3 * i] * gi[3 * j]",
     "test_bruteforce_equals_pointwise_definition"),
    ("Cartesian g' sign of the l R / r^(l+1) term",
     "double g1 = dR / rl - (double)l * R / (rl * r);", "double g1 = dR / rl + (double)l * R / (rl * r);",
     "test_cartesian_basis_equals_spherical"),
    ("tau term factor 1/2 dropped",
     "double tt = tau ? wp * vtau[p] * 0.5 * gg : 0.0;", "double tt = tau ? wp * vtau[p] * gg : 0.0;",
     "test_tau_term_pins"),
    # density (Eq. Density), its gradient and Hessian
    ("density reads P_ii instead of P_ij",
     "double t = phi[a] * row[idx[b]] * phi[b];", "double t = phi[a] * row[idx[a]] * phi[b];",
     "test_symmetry_trace_and_positivity"),
    ("electron count without the weights",
     "if (w) neu_add(&nes, &nec, w[p] * n[p]);", "if (w) neu_add(&nes, &nec, n[p]);",
     "test_symmetry_trace_and_positivity"),
    ("density gradient factor 2 dropped",
     "double t = 2.0 * grad[3 * a + c] * row[idx[b]] * phi[b];", "double t = grad[3 * a + c] * row[idx[b]] * phi[b];",
     "test_density_gradient_matches_finite_differences"),
    ("density Hessian loses a gradient product",
     "pij * grad[3 * a + ib] * grad[3 * b + ia], pij * phi[a] * hs[6 * b + k]}",
     "0.0 * grad[3 * a + ib] * grad[3 * b + ia], pij * phi[a] * hs[6 * b + k]}",
     "test_density_hessian_differences_and_rank_one"),
    # error denominators (the scale of every parity bar)
    ("H magnitude sum drops the kinetic term",
     "neu_add(&A[e], &Ac[e], fabs(tv) + fabs(tk) + fabs(tt));", "neu_add(&A[e], &Ac[e], fabs(tv) + fabs(tt));",
     "test_error_denominators"),
    ("density magnitude sum takes signed terms",
     "neu_add(&ds, &dc, fabs(t));", "neu_add(&ds, &dc, t);",
     "test_error_denominators"),
    ("gradient magnitude sum takes signed terms",
     "neu_add(&ds, &de, fabs(t));", "neu_add(&ds, &de, t);",
     "test_error_denominators"),
    ("density Hessian magnitude sum takes signed terms",
     "neu_add(&dv, &de, fabs(t[u]));", "neu_add(&dv, &de, t[u]);",
     "test_density_hessian_differences_and_rank_one"),
    # local Pulay terms
    ("Pulay magnitude sums take signed terms",
     "if (AM) AM[e] += fabs(tm);", "if (AM) AM[e] += tm;",
     "test_pulay_forces_routes_and_fixed_grid_derivatives"),
    ("Pulay force: sign of the q term",
     "+ 2.0 * wp * dRphi * qr[idx[b]] * phi[b];", "- 2.0 * wp * dRphi * qr[idx[b]] * phi[b];",
     "test_pulay_forces_routes_and_fixed_grid_derivatives"),
    ("Pulay matrices: Laplacian takes yz for zz",
     "hs[6 * b + 5]) + vp * phi[b];\n        for (int c = 0; c < 3; c++)",
     "hs[6 * b + 4]) + vp * phi[b];\n        for (int c = 0; c < 3; c++)",
     "test_pulay_forces_routes_and_fixed_grid_derivatives"),
    ("Pulay force: d/dR_at phi = +grad phi",
     "double dRphi = -grad[3 * a + c];", "double dRphi = grad[3 * a + c];",
     "test_pulay_forces_routes_and_fixed_grid_derivatives"),
    ("Pulay matrices: S^c takes phi_i for phi_j",
     "double ts = wp * (grad[3 * a + c] * phi[b]);", "double ts = wp * (grad[3 * a + c] * phi[a]);",
     "test_pulay_forces_routes_and_fixed_grid_derivatives"),
    # periodic h(k) (Eq. HamPeriodic with the Bloch basis)
    ("Bloch functions not conjugated on the left",
     "double re = cr[i] * cr[j] + ci[i] * ci[j], im = cr[i] * ci[j] - ci[i] * cr[j];",
     "double re = cr[i] * cr[j] - ci[i] * ci[j], im = cr[i] * ci[j] + ci[i] * cr[j];",
     "test_hermitian_time_reversal_and_reciprocal_shift"),
    ("translation added instead of subtracted along x",
     "double q[3] = {pts[3 * p] - T[0],", "double q[3] = {pts[3 * p] + T[0],",
     "test_supercell_spectrum_is_union_of_k_spectra"),
    ("periodic kinetic factor 1/2 dropped",
     "tr += 0.5 * wp * re; ti += 0.5 * wp * im;", "tr += wp * re; ti += wp * im;",
     "test_bloch_sum_of_the_image_system_hamiltonian"),
    ("Bloch phase e^{-ik.T} for e^{ik.T}",
     "double ph = k[0] * T[0] + k[1] * T[1] + k[2] * T[2];", "double ph = -(k[0] * T[0] + k[1] * T[1] + k[2] * T[2]);",
     "test_bloch_sum_of_the_image_system_hamiltonian"),
    ("periodic kinetic magnitude sum loses its 1/2",
     "ta += 0.5 * fabs(wp) * mag;", "ta += fabs(wp) * mag;",
     "test_periodic_error_denominators"),
    # partition and relevance (Sec. 3.3.1, 3.3.2)
    ("tie between equal extents goes to y",
     "if (ext[1] > ext[ax]) ax = 1;", "if (ext[1] >= ext[ax]) ax = 1;",
     "test_first_cut_is_a_plane_on_largest_axis_and_ties_pick_x"),
    ("left part rounded up",
     "int64_t nL = (n * kL) / k;", "int64_t nL = (n * kL + k - 1) / k;",
     "test_partition_left_part_is_rounded_down"),
    ("sort key: index ties reversed",
     "return (x->idx > y->idx) - (x->idx < y->idx);", "return (x->idx < y->idx) - (x->idx > y->idx);",
     "test_equal_coordinates_keep_index_order"),
    ("relevance boundary not strict",
     "if (minr2 < rc * rc) {", "if (minr2 <= rc * rc) {",
     "test_relevance_boundary_is_strict"),
    ("relevance looks at the batch's first point only",
     "for (int64_t q = offsets[b]; q < offsets[b + 1]; q++) {", "for (int64_t q = offsets[b]; q < offsets[b] + 1; q++) {",
     "test_relevance_matches_brute_force_scan"),
    ("relevance distance counts dy twice",
     "double r2 = (dx * dx + dy * dy) + dz * dz;", "double r2 = (dx * dx + dy * dy) + dy * dy;",
     "test_relevance_matches_brute_force_scan"),
]


def _slug(name):
    return re.sub(r"[^a-z0-9]+", "_", name.lower()).strip("_")[:60]


def _run_mutant(src, m):
    name, old, new, _ = m
    tag = _slug(name)
    c_path, so_path = OUT / f"{tag}.c", OUT / f"{tag}.so"
    c_path.write_text(src.replace(old, new, 1))
    subprocess.run(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
                    "-D_DEFAULT_SOURCE", str(c_path), "-o", str(so_path), "-lm"], check=True, capture_output=True)
    # one BLAS thread per run: the runs themselves go in parallel, one per core
    env = dict(os.environ, NAO_ORACLE_LIB=str(so_path), PYTHONDONTWRITEBYTECODE="1", OMP_NUM_THREADS="1",
               OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-rf", "-p", "no:cacheprovider", "-m", "not gpu", *PINS],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    failed = set(re.findall(r"^FAILED \S+?::(\w+)", r.stdout, flags=re.M))
    return r.returncode, failed, r.stdout[-2000:]


@pytest.mark.slow
def test_every_planted_mistake_is_caught():
    src = SRC.read_text()
    for name, old, new, _ in MUTANTS:
        assert src.count(old) == 1, f"mutant '{name}': its text must occur exactly once in oracle.c"
        assert old != new
    OUT.mkdir(parents=True, exist_ok=True)
    try:
        with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
            results = list(ex.map(lambda m: _run_mutant(src, m), MUTANTS))
    finally:
        shutil.rmtree(OUT, ignore_errors=True)
    problems = []
    for (name, _, _, pin), (rc, failed, tail) in zip(MUTANTS, results):
        print(f"{name}: {len(failed)} pins fail ({', '.join(sorted(failed))})")
        if rc != 1 or not failed:
            problems.append(f"'{name}' survived (pytest exit {rc}):\n{tail}")
        elif pin not in failed:
            problems.append(f"'{name}' is caught, but not by {pin}: {sorted(failed)}")
    assert not problems, "\n".join(problems)
