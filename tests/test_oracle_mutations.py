"""Planted mistakes in the oracle (on the CPU): each plausible error — a wrong sign, a dropped
term, a wrong coefficient, a wrong stage time, a transposed index — is written into a temporary
copy of the C oracle, and at least one pin of tests/test_oracle_pins.py must fail with it.
The clause-by-clause coefficients of Eq. kpath get three: the two segment weights swapped, the
partial sum H_k missing its own clause, and the two segments meeting at s = k/m both counted.
Four more go into the step-size control (the acceptance test, the halving, the restart of a
rejected start-up, the PEC evaluation time) and three into the XY start (the highest eigenvector,
the neighbouring sector, the first excited energy), each caught by its own pins.
This shows the pins are sharp enough to catch mistakes anywhere in the oracle."""
import ctypes as C
import os
import subprocess

import pytest

import test_oracle_cbc_pins as cbc
import test_oracle_pins as pins
from oracle import oracle as O

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "aqc_oracle.c")

MUTATIONS = {
    "sigma_y_sign": ("*re = -i * sign;", "*re = i * sign;"),
    "indicator_penalty": ("return k == 1 ? 0.0 : 1.0;", "return k == 1 ? 1.0 : 0.0;"),
    "scatter_at_source": ("jb->out[2 * zout] += c * re;", "jb->out[2 * z] += c * re;"),
    "minus_i_sign": ("f[2 * z] = tmp[2 * z + 1];", "f[2 * z] = -tmp[2 * z + 1];"),
    "rk4_stage_time": ("if (deriv(H, sc, t + 0.5 * h, ys, k, tmp, N, nthreads)) goto fail;",
                       "if (deriv(H, sc, t + h, ys, k, tmp, N, nthreads)) goto fail;"),
    "rk4_weight": ("psi[i] += (h / 6.0) * acc[i];", "psi[i] += (h / 5.0) * acc[i];"),
    "predictor_dropped_term": ("+ 37.0 * fn2[i] - 9.0 * fn3[i]);", "+ 37.0 * fn2[i]);"),
    "corrector_coefficient": ("+ 19.0 * fn[i] - 5.0 * fn1[i]", "+ 18.0 * fn[i] - 5.0 * fn1[i]"),
    "smoothstep": ("s = 3.0 * tau * tau - 2.0 * tau * tau * tau;", "s = 3.0 * tau * tau - 2.0 * tau * tau;"),
    # clause-by-clause coefficients of Eq. kpath
    "kpath_weights_swapped": ("return (1.0 - sk) * (double)in_prev + sk * (double)in_cur;",
                              "return sk * (double)in_prev + (1.0 - sk) * (double)in_cur;"),
    "kpath_partial_sum_index": ("int in_cur = (k <= m - 1) && (j <= k);", "int in_cur = (k <= m - 1) && (j < k);"),
    "kpath_segments_summed": (
        "    if (!(sk >= 0.0 && sk < 1.0)) continue;",
        "    if (!(sk >= 0.0 && sk <= 1.0)) continue;\n"
        "    if (sk == 1.0 && k < m) { double sn = sk - 1.0; int pn = (j <= k); int cn = (k + 1 <= m - 1) && (j <= k + 1);\n"
        "      return (1.0 - sk) * (double)((k - 1 >= 1) && (j <= k - 1)) + sk * (double)((k <= m - 1) && (j <= k))\n"
        "             + (1.0 - sn) * (double)pn + sn * (double)cn; }"),
}

PINS = [
    lambda: pins.test_hpsi_matches_dense(4),
    lambda: pins.test_final_hamiltonian_ground_state_brute_force(8, 1),
    pins.test_golden_bit_order_and_clauses,
    pins.test_rk4_startup_is_fourth_order_taylor,
    lambda: pins.test_constant_hamiltonian_matches_exponential(3),
    pins.test_landau_zener,
    lambda: pins.test_product_state_time_dependent(0),
    lambda: pins.test_product_state_time_dependent(1),
    pins.test_x_driver_ground_state_and_spectrum,
    pins.test_c_schedule_weights_closed_form,
    lambda: pins.test_diagonal_hamiltonian_phases(1),
    lambda: cbc.test_segments_interpolate_partial_sums(1),
    lambda: cbc.test_one_segment_on_step_grids(7, 2940),
]


def _mutant(tmp_path, name, table=None):
    old, new = (table or MUTATIONS)[name]
    src = open(SRC).read()
    assert src.count(old) >= 1, name
    mut = src.replace(old, new, 1)
    c_path = tmp_path / f"{name}.c"
    so_path = tmp_path / f"{name}.so"
    c_path.write_text(mut)
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", str(so_path), str(c_path),
                           "-lpthread", "-lm"])
    return str(so_path)


def _bind(path):
    lib = C.CDLL(path)
    lib.or_hpsi.argtypes = [C.POINTER(O._Ham), C.POINTER(C.c_double), C.c_void_p, C.c_void_p, C.c_int]
    lib.or_hpsi.restype = C.c_int
    lib.or_propagate.argtypes = [C.POINTER(O._Ham), C.POINTER(O._Sched), C.c_int64, C.c_int64, C.c_void_p,
                                 C.POINTER(O._Stats), C.c_int]
    lib.or_propagate.restype = C.c_int
    lib.or_hpsi_at.argtypes = [C.POINTER(O._Ham), C.POINTER(C.c_double), C.c_void_p, C.c_int64, C.c_void_p,
                               C.c_void_p]
    lib.or_hpsi_at.restype = C.c_int
    lib.or_weights.argtypes = [C.POINTER(O._Sched), C.c_double, C.POINTER(C.c_double)]
    lib.or_weights.restype = None
    lib.or_propagate_adaptive.argtypes = [C.POINTER(O._Ham), C.POINTER(O._Sched), C.c_double, C.c_double, C.c_int,
                                          C.c_double, C.c_int64, C.c_void_p, C.POINTER(O._AStats),
                                          C.POINTER(O._Segment), C.c_int64, C.c_void_p, C.c_int64, C.c_int]
    lib.or_propagate_adaptive.restype = C.c_int
    return lib


def test_unmutated_oracle_passes_the_battery():
    O._load()
    for p in PINS:
        p()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_is_caught(tmp_path, monkeypatch, name):
    lib = _bind(_mutant(tmp_path, name))
    monkeypatch.setattr(O, "_lib", lib)
    failed = []
    for i, p in enumerate(PINS):
        try:
            p()
        except AssertionError:
            failed.append(i)
        except RuntimeError:
            failed.append(i)
    assert failed, f"no pin caught the planted mistake {name}"


# Planted mistakes in the oracle's Python builders of the XY / XYZ algorithms (Sec. III.A.2-3):
# the function's own source with one substitution, run in the oracle module's namespace.
PY_MUTATIONS = {
    "xy_yy_sign": ("add_xy_driver", "H.add_term(group, m, m, -omega * v / 2.0)",
                   "H.add_term(group, m, m, omega * v / 2.0)"),
    "xy_identity_prefactor": ("add_xy_driver", "3.0 * len(clauses) * omega", "2.0 * len(clauses) * omega"),
    "xyz_zz_dropped": ("add_xyz_driver", "H.add_term(group, 0, m, -a)  # Z_i Z_j", "pass"),
    "xyz_pair_weight": ("add_xyz_driver", "a = omega * v / 2.0", "a = omega * v"),
    "pair_counts_with_self_pairs": ("clause_pair_counts", "for y in range(x + 1, 3):", "for y in range(x, 3):"),
    "dicke_normalisation": ("dicke_state", "1.0 / math.sqrt(math.comb(n, k))", "1.0 / math.comb(n, k)"),
}


def _xy_pins():
    import test_oracle_xy_pins as xy

    return [
        lambda: xy.test_drivers_on_basis_states(1),
        xy.test_dicke_states_are_xyz_ground_states,
        lambda: xy.test_paths_conserve_hamming_weight("xy"),
    ]


def test_unmutated_xy_builders_pass_their_pins():
    for p in _xy_pins():
        p()


@pytest.mark.parametrize("name", sorted(PY_MUTATIONS))
def test_planted_mistake_in_xy_builders_is_caught(monkeypatch, name):
    import inspect
    import textwrap

    func, old, new = PY_MUTATIONS[name]
    src = textwrap.dedent(inspect.getsource(getattr(O, func)))
    assert src.count(old) == 1, name
    ns = dict(vars(O))
    exec(compile(src.replace(old, new), O.__file__, "exec"), ns)
    monkeypatch.setattr(O, func, ns[func])
    failed = []
    for i, p in enumerate(_xy_pins()):
        try:
            p()
        except (AssertionError, RuntimeError, ValueError):
            failed.append(i)
    assert failed, f"no pin caught the planted mistake {name}"


# Planted mistakes in the step-size control (or_propagate_adaptive, reading of Sec. I.B): the
# acceptance test, the halving, the restart of a segment whose first PEC step is rejected, and
# the time of the PEC evaluation; each must be caught by a pin of test_oracle_adaptive_pins.py.
ADAPTIVE_MUTATIONS = {
    "adaptive_accepts_twice_the_tolerance": ("if (!(est <= lim)) {", "if (!(est <= 2.0 * lim)) {"),
    "adaptive_quarters_instead_of_halving": ("hp = 0.5 * h;", "hp = 0.25 * h;"),
    "adaptive_keeps_the_rejected_start_up": ("memcpy(psi, yseg, bytes);", ";"),
    "adaptive_pec_evaluation_time": ("if (deriv(H, sc, t0 + (double)(kk + 1) * h, p, fnew, tmp, N, nthreads))",
                                     "if (deriv(H, sc, t0 + (double)kk * h, p, fnew, tmp, N, nthreads))"),
}


def _adaptive_pins():
    import test_oracle_adaptive_pins as ad

    return [
        lambda: ad.test_no_rejection_is_the_fixed_grid_bit_for_bit(1),
        ad.test_unstable_start_is_rejected_down_to_a_stable_step,
        ad.test_every_accepted_estimate_is_within_tolerance,
    ]


def test_unmutated_step_control_passes_its_pins():
    O._load()
    for p in _adaptive_pins():
        p()


@pytest.mark.parametrize("name", sorted(ADAPTIVE_MUTATIONS))
def test_planted_mistake_in_step_control_is_caught(tmp_path, monkeypatch, name):
    lib = _bind(_mutant(tmp_path, name, ADAPTIVE_MUTATIONS))
    monkeypatch.setattr(O, "_lib", lib)
    failed = []
    for i, p in enumerate(_adaptive_pins()):
        try:
            p()
        except (AssertionError, RuntimeError):
            failed.append(i)
    assert failed, f"no pin caught the planted mistake {name}"


# Planted mistakes in the XY start (xy_sector_ground_state): the highest instead of the lowest
# eigenvector, and a neighbouring Hamming-weight sector.
GROUND_MUTATIONS = {
    "xy_ground_highest_eigenvector": ("v = V[:, 0]", "v = V[:, -1]"),
    "xy_ground_wrong_sector": ('if bin(z).count("1") == k], dtype=np.int64)',
                               'if bin(z).count("1") == k + 1], dtype=np.int64)'),
    "xy_ground_energy_of_the_first_excited_level": ("return float(lam[0]), psi", "return float(lam[1]), psi"),
}


def _ground_pins():
    import test_oracle_xy_pins as xy

    return [
        lambda: xy.test_xy_ground_state_against_the_hopping_block(8, 1),
        lambda: xy.test_xy_ground_state_on_the_complete_graph_is_dicke(5),
        xy.test_xy_ground_state_against_the_kronecker_matrix,
    ]


@pytest.mark.parametrize("name", sorted(GROUND_MUTATIONS))
def test_planted_mistake_in_the_xy_start_is_caught(monkeypatch, name):
    import inspect
    import textwrap

    old, new = GROUND_MUTATIONS[name]
    src = textwrap.dedent(inspect.getsource(O.xy_sector_ground_state))
    assert src.count(old) == 1, name
    ns = dict(vars(O))
    exec(compile(src.replace(old, new), O.__file__, "exec"), ns)
    monkeypatch.setattr(O, "xy_sector_ground_state", ns["xy_sector_ground_state"])
    failed = []
    for i, p in enumerate(_ground_pins()):
        try:
            p()
        except (AssertionError, RuntimeError, ValueError, IndexError):
            failed.append(i)
    assert failed, f"no pin caught the planted mistake {name}"
