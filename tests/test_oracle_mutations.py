"""The oracle's pins are not vacuous.  A copy of the oracle's C sources gets one planted mistake, the kind
a slip in writing it out would make: a wrong sign, a dropped term, a missing conjugate, a transposed
operand or index, too few iterations.  The copy is built into a library of its own, and the pins run
against it.  At least one pin must fail for every mistake.  CPU only; the mistakes live in the copies,
never in the oracle.  Every planted mistake keeps all memory accesses in bounds (the copies run in this
process)."""
from __future__ import annotations

import os
import shutil

import pytest

import oracle
from tests import test_oracle_pins as P

ORACLE_DIR = os.path.dirname(os.path.abspath(oracle.__file__))

# (name, file, text as written, text with the planted mistake, pins that must notice)
MUTATIONS = [
    ("jacobi rotation sign", "eigh.c",
     "if (mp_sign(&tau) < 0) mp_neg(&t, &t);", "if (mp_sign(&tau) > 0) mp_neg(&t, &t);",
     [P.test_eigh_2x2_closed_form, lambda: P.test_eigh_exact_known_spectrum(6, 2)]),
    ("jacobi eigenvector update with the wrong phase", "eigh.c",
     "cmp_mul(&u2, &z1, &y); cmp_sub(&np_, &u1, &u2);\n          cmp_mul(&u1, &z2, &x); cmp_scale(&u2, &y, &c); "
     "cmp_add(&nq, &u1, &u2);\n          v[IDX",
     "cmp_mul(&u2, &z2, &y); cmp_sub(&np_, &u1, &u2);\n          cmp_mul(&u1, &z2, &x); cmp_scale(&u2, &y, &c); "
     "cmp_add(&nq, &u1, &u2);\n          v[IDX",
     [P.test_eigh_eigenvectors_of_distinct_spectrum_match_exact_columns, lambda: P.test_eigh_exact_known_spectrum(6, 2)]),
    ("jacobi diagonal update dropped", "eigh.c",
     "mp_add(&a[IDX(q, q, n)].re, &a[IDX(q, q, n)].re, &tb);", "",
     [P.test_eigh_2x2_closed_form, lambda: P.test_eigh_exact_known_spectrum(6, 2)]),
    ("eigenvalues sorted ascending", "eigh.c",
     "mp_cmp(&a[IDX(order[j], order[j], n)].re, &a[IDX(k, k, n)].re) < 0",
     "mp_cmp(&a[IDX(order[j], order[j], n)].re, &a[IDX(k, k, n)].re) > 0",
     [lambda: P.test_eigh_exact_known_spectrum(6, 2)]),
    ("residual without the eigenvalue term", "eigh.c",
     "cmp_scale(&t, &vv[IDX(i, c, n)], &l); cmp_sub(&s, &s, &t);", "cmp_scale(&t, &vv[IDX(i, c, n)], &l);",
     [P.test_residual_and_orthonormality_match_exact_values]),
    ("orthonormality without the conjugate", "eigh.c",
     "cmp_mul_conj(&t, &vv[IDX(i, d, n)], &vv[IDX(i, c, n)])", "cmp_mul(&t, &vv[IDX(i, d, n)], &vv[IDX(i, c, n)])",
     [P.test_residual_and_orthonormality_match_exact_values]),
    ("multiply drops the lowest limb of one operand", "mp.c",
     "for (int j = 0; j < MPL; ++j) {\n      u128 t = (u128)a->m[i] * b->m[j]",
     "for (int j = 1; j < MPL; ++j) {\n      u128 t = (u128)a->m[i] * b->m[j]",
     [lambda: P.test_mp_scalar_ops_match_exact_rationals("mul")]),
    ("reciprocal with one Newton step", "mp.c",
     "for (int it = 0; it < 5; ++it) {                   /* x <- x + x (1 - b x)",
     "for (int it = 0; it < 1; ++it) {                   /* x <- x + x (1 - b x)",
     [lambda: P.test_mp_scalar_ops_match_exact_rationals("div")]),
    ("addition carry without the exponent step", "mp.c",
     "x[MPL + 1] = 0; e += 1;", "x[MPL + 1] = 0;",
     [lambda: P.test_mp_scalar_ops_match_exact_rationals("add")]),
    ("inverse square root with one Newton step", "mp.c",
     "for (int it = 0; it < 5; ++it) {                   /* y <- y + y (1 - aa y^2) / 2 */",
     "for (int it = 0; it < 1; ++it) {                   /* y <- y + y (1 - aa y^2) / 2 */",
     [P.test_mp_sqrt_matches_integer_sqrt]),
    ("two-qubit gate with the qubit roles swapped", "statevec.c",
     "size_t idx[4] = {x, x | bj, x | bi, x | bi | bj};", "size_t idx[4] = {x, x | bi, x | bj, x | bi | bj};",
     [P.test_statevector_gates_on_basis_states]),
    ("two-qubit gate applied transposed", "statevec.c",
     "cmp_mul(&t, &g[r * 4 + c], &in[c]);", "cmp_mul(&t, &g[c * 4 + r], &in[c]);",
     [P.test_statevector_gates_on_basis_states]),
    ("one-qubit gate on the mirrored site", "statevec.c",
     "cmp_t g[4]; load_mat(g, U, 2, w);\n  size_t bit = (size_t)1 << (h->n - 1 - site);",
     "cmp_t g[4]; load_mat(g, U, 2, w);\n  size_t bit = (size_t)1 << site;",
     [P.test_statevector_gates_on_basis_states]),
    ("controlled gate ignores the control value", "statevec.c",
     "ok = bit == ctrl[l];", "ok = 1;",
     [P.test_statevector_gates_on_basis_states]),
    ("state norm without the squares", "statevec.c",
     "for (size_t x = 0; x < h->dim; ++x) { cmp_abs2(&t, &h->psi[x]); mp_add(&acc, &acc, &t); }",
     "for (size_t x = 0; x < h->dim; ++x) { t = h->psi[x].re; mp_add(&acc, &acc, &t); }",
     [P.test_statevector_ghz_and_norm_and_reversibility]),
    ("MPS amplitudes weight every branch by the first Schmidt value", "statevec.c",
     "if (lw) cmp_scale(&u, &u, &lw[a]);", "if (lw) cmp_scale(&u, &u, &lw[0]);",
     [P.test_mps_amplitudes_ghz]),
    ("canonical defect without the conjugate", "statevec.c",
     "cmp_mul_conj(&t, x, y);                        /* conj(x) y */", "cmp_mul(&t, x, y);",
     [lambda: P.test_mps_site_defect_exact_isometries(3, 5, 2)]),
    ("canonical defect weights not squared", "statevec.c",
     "mp_mul(&wt[k], &t, &t);", "wt[k] = t;",
     [lambda: P.test_mps_site_defect_exact_isometries(3, 5, 2)]),
    ("Schmidt values: right Gram matrix summed over the wrong index", "statevec.c",
     "cmp_mul_conj(&t, &h->psi[l * R + b], &h->psi[l * R + a])", "cmp_mul_conj(&t, &h->psi[b * R + l], &h->psi[a * R + l])",
     [lambda: P.test_statevector_footnote_schmidt_values_u_is_z(8), P.test_footnote_golden_schmidt_values]),
    ("jacobi stops at 2^-100 of the norm", "eigh.c",
     "mp_ldexp(&tol, &fro, -300);", "mp_ldexp(&tol, &fro, -100);",
     [lambda: P.test_eigh_exact_known_spectrum(6, 2), P.test_eigh_2x2_closed_form]),
    ("non-Hermitian input accepted", "eigh.c",
     "free(a); free(v); free(vs); free(lam); free(order); return 1;", "(void)0;",
     [P.test_eigh_rejects_non_hermitian]),
    ("Vidal tensors divided by the right weight only", "statevec.c",
     "mp den; mp_mul(&den, &L[l][al], &L[l + 1][be]);", "mp den = L[l + 1][be];",
     [P.test_statevector_vidal_form_reproduces_the_state]),
    ("Vidal right Schmidt vectors without the conjugate", "statevec.c",
     "for (size_t r = 0; r < Rd; ++r) cmp_conj(&V[c][r + Rd * q], &e[r]);",
     "for (size_t r = 0; r < Rd; ++r) V[c][r + Rd * q] = e[r];",
     [P.test_statevector_vidal_form_reproduces_the_state]),
    ("MPS expectation with the left weights not squared", "statevec.c",
     "else { mp t; mp_from_words(&t, lam + (loff + k) * w, w); mp_mul(&wl[k], &t, &t); }",
     "else { mp_from_words(&wl[k], lam + (loff + k) * w, w); }",
     [P.test_one_qubit_expectation_values_two_ways]),
    ("state-vector expectation without the conjugate", "statevec.c",
     "cmp_mul_conj(&t, &a0, &r0); cmp_add(&acc, &acc, &t);", "cmp_mul(&t, &a0, &r0); cmp_add(&acc, &acc, &t);",
     [P.test_one_qubit_expectation_values_two_ways]),
    ("one-sided Jacobi inner product without the conjugate", "svd.c",
     "cmp_mul_conj(&t, &a[IX(i, p, m)], &a[IX(i, q, m)]); cmp_add(&g, &g, &t);",
     "cmp_mul(&t, &a[IX(i, p, m)], &a[IX(i, q, m)]); cmp_add(&g, &g, &t);",
     [lambda: P.test_svd_of_exact_construction(5, 3, 3)]),
    ("one-sided Jacobi rotations not accumulated in V", "svd.c",
     "for (int pass = 0; pass < 2; ++pass) {", "for (int pass = 0; pass < 1; ++pass) {",
     [lambda: P.test_svd_of_exact_construction(5, 3, 3)]),
    ("two-product Vidal form: Cholesky off-diagonal not divided by the pivot", "statevec.c",
     "cmp_t q01; mp_div(&q01.re, &G->x[0][1].re, &q00); mp_div(&q01.im, &G->x[0][1].im, &q00);",
     "cmp_t q01 = G->x[0][1];",
     [P.test_two_product_vidal_form_matches_the_state_vector]),
    ("two-product Vidal tensors without the term coefficients", "statevec.c",
     "cmp_mul(&u, &c[t], &ul);", "u = ul;",
     [P.test_two_product_vidal_form_matches_the_state_vector]),
    ("gate update: theta without the middle weights", "mpsgate.c",
     "      cmp_scale(&x, &x, &wc[be]);\n", "",
     [P.test_mps_gate_update_matches_the_state_vector]),
    ("gate update: right tensor without the conjugate", "mpsgate.c",
     "cmp_t u; cmp_conj(&u, &Vm[(size_t)(s * d + ga) + (size_t)j * C]);",
     "cmp_t u = Vm[(size_t)(s * d + ga) + (size_t)j * C];",
     [P.test_mps_gate_update_matches_the_state_vector]),
    ("gate update: kept weights not renormalised", "mpsgate.c",
     "mp t; mp_div(&t, &sg[order[be]], &nrm);", "mp t = sg[order[be]];",
     [P.test_mps_gate_update_matches_the_state_vector, P.test_mps_gate_update_truncation_keeps_the_schmidt_fidelity]),
    ("sampling marginals without the Schmidt weights", "mpsgate.c",
     "if (k < n - 1) { mp_from_words(&wt, lam + (lo + be) * w, w); mp_mul(&wt, &wt, &wt); mp_mul(&m2, &m2, &wt); }",
     "(void)wt;", [P.test_mps_sampling_follows_the_born_rule]),
    ("conjugate-transpose product without the conjugate", "products.c",
     "if (opA) cmp_mul_conj(&t,", "if (opA) cmp_mul(&t,",
     [P.test_matmul_matches_exact_rationals]),
    ("plain product reads A transposed", "products.c",
     "else cmp_mul(&t, &a[(size_t)i + (size_t)l * ar]", "else cmp_mul(&t, &a[(size_t)l + (size_t)i * ar]",
     [P.test_matmul_matches_exact_rationals]),
]


@pytest.mark.parametrize("name,fname,old,new,pins", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_fails_a_pin(tmp_path, monkeypatch, name, fname, old, new, pins):
    for f in os.listdir(ORACLE_DIR):
        if f.endswith((".c", ".h")):
            shutil.copy(os.path.join(ORACLE_DIR, f), tmp_path / f)
    src = (tmp_path / fname).read_text()
    assert src.count(old) == 1, f"the text to change is not unique in {fname}: {old!r}"
    (tmp_path / fname).write_text(src.replace(old, new))
    lib = oracle.load_library(oracle.compile_library(str(tmp_path), str(tmp_path / "mutant.so")))
    monkeypatch.setattr(oracle, "_lib", lib)
    failed = []
    for pin in pins:
        try:
            pin()
        except (AssertionError, RuntimeError, ValueError, ZeroDivisionError, pytest.fail.Exception):
            failed.append(pin)
    assert failed, f"no pin noticed the planted mistake: {name}"


def test_unchanged_copy_passes_the_same_pins(tmp_path, monkeypatch):
    """The harness itself: a copy without a planted mistake passes every pin used above."""
    for f in os.listdir(ORACLE_DIR):
        if f.endswith((".c", ".h")):
            shutil.copy(os.path.join(ORACLE_DIR, f), tmp_path / f)
    lib = oracle.load_library(oracle.compile_library(str(tmp_path), str(tmp_path / "copy.so")))
    monkeypatch.setattr(oracle, "_lib", lib)
    seen = set()
    for *_, pins in MUTATIONS:
        for pin in pins:
            if id(pin) not in seen:
                seen.add(id(pin))
                pin()
