"""The pins catch plausible mistakes in the oracle.

Each case plants one mistake in the FP64 oracle, on the CPU, through
``monkeypatch`` (a dropped term, a wrong sign or index, a transposed operand, a
wrong convention). The oracle calls its own steps through module globals, so
the mistake reaches every function that uses the step. The pins named for the
case then run against the mutated oracle, and at least one of them must fail.
A mutation that no pin catches would be a part of the oracle that nothing
outside the oracle fixes.
"""
import numpy as np
import pytest

import oracle as orc
import oracle.oracle as impl
import test_oracle_pins as pins


def _fails(fn) -> bool:
    try:
        fn()
    except Exception:      # an assertion, or a mistake that breaks the computation itself
        return True
    return False


def _patch(mp, name, make):
    """Replace the oracle's step <name> by make(original), in the module that
    defines it (so that its other functions call the mutated step) and in the
    package namespace the pins call."""
    mutated = make(getattr(impl, name))
    mp.setattr(impl, name, mutated)
    if hasattr(orc, name):
        mp.setattr(orc, name, mutated)


def _cheb_plus(orig):
    def basis_values(kind, lam, lam_s, p):
        out = orig(kind, lam, lam_s, p)
        if kind == orc.BASIS_CHEB_LOG:
            u = out[:, 1].copy() if p > 1 else None
            for m in range(2, p):
                out[:, m] = 2.0 * u * out[:, m - 1] + out[:, m - 2]   # sign of T_{m-2} flipped
        return out
    return basis_values


def _cholesky_last_pivot(orig):
    def cholesky(A):
        L = orig(A)
        if L.shape[0] > 1:
            L[-1, -1] = np.sqrt(np.asarray(A, dtype=np.float64)[-1, -1])   # update of the last pivot dropped
        return L
    return cholesky


def _argmin_last(orig):
    def argmin_first(values):
        best, best_t = np.inf, -1
        for t, v in enumerate(values):
            if np.isfinite(v) and v <= best:                          # ties go to the last index
                best, best_t = v, t
        return best_t
    return argmin_first


def _unusable_eps(orig):
    def diag_unusable(diag):
        m = float(np.max(np.abs(diag))) if diag.size else 0.0
        thr = np.finfo(np.float64).eps * m                            # the 1e3 factor dropped
        return bool(np.any(diag <= 0.0) or np.any(np.abs(diag) <= thr))
    return diag_unusable


class _NumpyWith:
    """numpy with some functions replaced, for a mistake inside an oracle
    function that calls numpy directly."""

    def __init__(self, **over):
        self._over = over

    def __getattr__(self, name):
        return self._over[name] if name in self._over else getattr(np, name)


MUTATIONS = {
    "holdout error drops the last output column": (
        lambda mp: _patch(mp, "holdout_sse",
                          lambda o: lambda Xv, Yv, W: o(Xv, Yv[:, :-1], W[:, :-1]) if Yv.shape[1] > 1 else 0.0),
        [pins.test_holdout_sse_direct_and_expansion, pins.test_exact_cv_matches_independent_library_pipeline]),
    "holdout error not divided by the output count": (
        lambda mp: _patch(mp, "holdout_sse", lambda o: lambda Xv, Yv, W: o(Xv, Yv, W) * Yv.shape[1]),
        [pins.test_exact_cv_matches_independent_library_pipeline]),
    "Cholesky drops the last pivot's update": (
        lambda mp: _patch(mp, "cholesky", _cholesky_last_pivot),
        [lambda: pins.test_cholesky_residual_and_structure(7), pins.test_cholesky_matches_library]),
    "forward substitution with the transposed factor": (
        lambda mp: _patch(mp, "forward", lambda o: impl.backward),
        [pins.test_triangular_solves_match_library, pins.test_ridge_matches_augmented_least_squares]),
    "back substitution with the untransposed factor": (
        lambda mp: _patch(mp, "backward", lambda o: impl.forward),
        [pins.test_triangular_solves_match_library, pins.test_ridge_matches_augmented_least_squares]),
    "normal equations leave out one row too many": (
        lambda mp: _patch(mp, "normal_blocks",
                          lambda o: lambda X, Y, s0=0, s1=0: o(X, Y, s0, s1 + 1 if s1 > s0 else s1)),
        [pins.test_normal_blocks_leave_out_rows]),
    "lambda grid spaced linearly": (
        lambda mp: _patch(mp, "lambda_grid", lambda o: lambda tau, q, lo, hi: tau * np.linspace(lo, hi, q)),
        [pins.test_sample_indices_and_grid, pins.test_exact_cv_matches_independent_library_pipeline]),
    "sample indices rounded down": (
        lambda mp: _patch(mp, "sample_indices",
                          lambda o: lambda q, g: [i * (q - 1) // (g - 1) for i in range(g)] if g > 1 else [0]),
        [pins.test_sample_indices_and_grid]),
    "Chebyshev recurrence with the wrong sign": (
        lambda mp: _patch(mp, "basis_values", _cheb_plus),
        [pins.test_chebyshev_basis_matches_library]),
    "basis derivative without the 1/lambda of the chain rule": (
        lambda mp: _patch(mp, "basis_derivs",
                          lambda o: lambda kind, lam, lam_s, p: o(kind, lam, lam_s, p) * np.atleast_1d(lam)[:, None]),
        [pins.test_basis_derivatives_match_finite_differences,
         lambda: pins.test_holdout_gradient_matches_central_differences(False, orc.BASIS_CHEB_LOG)]),
    "fit without the inverse of V^T V": (
        lambda mp: _patch(mp, "lstsq", lambda o: lambda V, T: np.asarray(V).T @ np.asarray(T)),
        [pins.test_lstsq_matches_library_and_pseudoinverse,
         lambda: pins.test_fit_reproduces_polynomials(orc.BASIS_MONO)]),
    "interpolation drops the highest-degree term": (
        lambda mp: _patch(mp, "eval_poly", lambda o: lambda phi, Theta: o(np.asarray(phi)[:-1], np.asarray(Theta)[:-1])),
        [pins.test_pichol_equals_exact_cv_when_every_lambda_is_a_node]),
    "vectorisation of the transposed factor": (
        lambda mp: _patch(mp, "vec_lower", lambda o: lambda L: o(np.ascontiguousarray(np.asarray(L).T))),
        [pins.test_vectorisation_round_trip]),
    "argmin takes the last of equal values": (
        lambda mp: _patch(mp, "argmin_first", _argmin_last),
        [pins.test_argmin_first_ties_and_inf]),
    "unusable-diagonal threshold without its 1e3 factor": (
        lambda mp: _patch(mp, "diag_unusable", _unusable_eps),
        [pins.test_unusable_diagonal_rule]),
    "trace scale divided by n instead of d": (
        lambda mp: _patch(mp, "trace_scale", lambda o: lambda X: o(X) * np.shape(X)[1] / np.shape(X)[0]),
        [pins.test_trace_scale]),
    "fold boundaries rounded up": (
        lambda mp: _patch(mp, "fold_offsets", lambda o: lambda n, k: [-((-f * n) // k) for f in range(k + 1)]),
        [pins.test_fold_offsets_partition_rows]),
    "MChol centre update in natural log": (
        lambda mp: mp.setattr(impl, "np", _NumpyWith(log10=np.log)),
        [pins.test_mchol_search_hand_traced]),
    "MChol runs one level too many": (
        lambda mp: _patch(mp, "mchol_levels", lambda o: lambda s, s_min: o(s, s_min) + 1),
        [pins.test_mchol_level_count, pins.test_mchol_search_hand_traced]),
    "exact hold-out error at twice the lambda": (
        lambda mp: _patch(mp, "holdout_exact_at",
                          lambda o: lambda X, Y, *, k, lams, folds=None: o(X, Y, k=k, lams=2.0 * np.asarray(lams),
                                                                          folds=folds)),
        [pins.test_exact_holdout_at_any_lambda_matches_eigen_closed_form,
         pins.test_pinrmse_matches_a_library_polynomial_fit_of_the_exact_errors]),
    "warm start without subtracting fold 0's fit at the warm samples": (
        lambda mp: _patch(mp, "warm_fit",
                          lambda o: lambda theta0, Vw, Tw, pw: o(theta0, Vw, Tw + Vw @ theta0, pw)),
        [lambda: pins.test_warm_start_with_every_sample_is_the_plain_fit("cheb_log"),
         pins.test_warm_start_interpolates_the_exact_factors_at_its_nodes]),
    "exact-system refinement with the wrong sign of lambda": (
        lambda mp: _patch(mp, "refine_exact_step",
                          lambda o: lambda Hf, lam, Lt, Bf, W: o(Hf, -lam, Lt, Bf, W)),
        [pins.test_exact_system_refinement_step_is_the_preconditioned_iteration,
         pins.test_exact_system_refinement_converges_to_exact_cv]),
    "NRMSE without its square roots": (
        lambda mp: _patch(mp, "nrmse", lambda o: lambda pred, target: o(pred, target) ** 2),
        [pins.test_nrmse_worked_by_hand, pins.test_nrmse_is_small_inside_a_well_sampled_range]),
    "gradient with the wrong sign": (
        lambda mp: _patch(mp, "_holdout_and_grad",
                          lambda o: lambda *a: (lambda e, de: (e, -de))(*o(*a))),
        [lambda: pins.test_holdout_gradient_matches_central_differences(False, orc.BASIS_CHEB_LOG)]),
}


@pytest.mark.parametrize("name", list(MUTATIONS))
def test_a_planted_mistake_fails_a_pin(monkeypatch, name):
    plant, checks = MUTATIONS[name]
    for check in checks:                    # every named pin passes on the oracle as it stands
        assert not _fails(check), f"pin fails before the mistake is planted ({name})"
    plant(monkeypatch)
    assert any(_fails(check) for check in checks), f"no pin catches: {name}"
