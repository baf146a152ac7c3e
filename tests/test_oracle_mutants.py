"""Planted mistakes: copies of the oracle, each with one plausible mistake
(a flipped sign, a dropped term, an off-by-one index, a wrong weight or
kernel width), built on the CPU; each must fail at least one pin of
test_oracle_pins.py, and the unchanged copy must pass them all."""
import importlib.util
import os

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# (name, text in oracle/mm_oracle.c, replacement)
MUTANTS = [
    ("phase_sign", "sum_add(&im, -delta[h] * sin(th));", "sum_add(&im, delta[h] * sin(th));"),
    ("phase_low_part_dropped", "double p_lo = fma(k, q_hi, -p_hi) + k * q_lo;", "double p_lo = 0.0;"),
    ("return_at_right_end_point", "rt[o] = t[h];", "rt[o] = t[h + 1];"),
    ("first_return_dropped", "for (int64_t h = off[i]; h + 1 < off[i + 1]; ++h) {\n      rt[o]",
     "for (int64_t h = off[i] + 1; h + 1 < off[i + 1]; ++h) {\n      rt[o]"),
    ("last_time_ignored_in_bounds", "if (t[h] > hi) hi = t[h];", "if (t[h] > hi && h + 1 < off[i + 1]) hi = t[h];"),
    ("dirichlet_weight_2N", "return 1.0 / (double)(2 * N + 1);", "return 1.0 / (double)(2 * N);"),
    ("fejer_textbook_weight", "(1.0 - ak / (double)N) / (double)(N + 1)",
     "(1.0 - ak / (double)(N + 1)) / (double)(N + 1)"),
    ("missing_conjugate", "(-k + N)); /* c^+_k(i)", "(k + N)); /* c^+_k(i)"),
    ("dirichlet_kernel_order", "sinpi_red((2.0 * Nd + 1.0) * y)", "sinpi_red((Nd + 1.0) * y)"),
    ("nyquist_factor_two", "floor(span / (2.0 * g))", "floor(span / g)"),
    ("es_half_width", "*alpha = ORC_PI * omega / (double)Mr;", "*alpha = ORC_PI * (double)msp / (double)Mr;"),
]


def _pins():
    spec = importlib.util.spec_from_file_location("_pins_for_mutants", os.path.join(HERE, "test_oracle_pins.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _battery(P):
    """Pins in rough order of cost (scipy-free, seconds in total)."""
    b = [
        (P.test_worked_example_sign_and_left_endpoint, {}),
        (P.test_c0_telescopes, {}),
        (P.test_hermitian_symmetry, {}),
        (P.test_shift_theorem, {}),
        (P.test_phase_exact_at_large_k, {}),
        (P.test_returns_count_and_left_endpoint, {}),
        (P.test_rescale_endpoints_and_bounds, {}),
        (P.test_nyquist_hand_example, {}),
        (P.test_single_return_weights, {"N": 5}),
        (P.test_dirichlet_N0_is_product_of_total_returns, {}),
        (P.test_dirichlet_on_exact_grid_is_realized_covariance, {}),
    ]
    for basis in ("dirichlet", "fejer"):
        b.append((P.test_bruteforce_triple_sum, {"basis": basis, "N": 2}))
        b.append((P.test_coefficient_route_equals_closed_kernel_route, {"basis": basis, "N": 7}))
        b.append((P.test_sigma_symmetric_psd_and_correlation, {"basis": basis}))
    for kernel in ("gauss", "kb", "es"):
        b.append((P.test_cpu_nufft_meets_requested_tolerance, {"kernel": kernel, "eps": 1e-6}))
    return b


def _build_variant(tmp_path, name, old, new):
    import oracle
    src = open(os.path.join(ROOT, "oracle", "mm_oracle.c")).read()
    if old is not None:
        assert src.count(old) >= 1, f"mutation site of {name} not found"
        src = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    c.write_text(src)
    so = tmp_path / f"{name}.so"
    oracle.compile_c(str(c), str(so))
    import ctypes
    L = ctypes.CDLL(str(so))
    oracle._declare(L)
    return L


def _failures(monkeypatch, L, stop_at_first):
    import oracle
    monkeypatch.setattr(oracle, "_lib", L)
    P = _pins()
    failed = []
    for fn, kw in _battery(P):
        try:
            fn(oracle, **kw)
        except AssertionError:
            failed.append(fn.__name__)
            if stop_at_first:
                break
    return failed


def test_unchanged_copy_passes_every_pin(tmp_path, monkeypatch):
    L = _build_variant(tmp_path, "unchanged", None, None)
    assert _failures(monkeypatch, L, stop_at_first=False) == []


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(tmp_path, monkeypatch, name, old, new):
    L = _build_variant(tmp_path, name, old, new)
    assert _failures(monkeypatch, L, stop_at_first=True), f"no pin catches {name}"
