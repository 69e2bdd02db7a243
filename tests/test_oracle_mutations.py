"""Planted mistakes in the oracle (CPU only) must each fail at least one pin.

Each mutation edits the oracle's source text, loads the edited copy as a module
and runs the pin battery of ``test_oracle_pins`` against it.
"""
import importlib.util
import os
import sys
import types

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ORACLE_SRC = os.path.join(os.path.dirname(HERE), "oracle", "ttals_oracle.py")

MUTATIONS = {
    # a wrong constant in the Householder reflection
    "reflector_factor": ("a[j:, j:] -= 2.0 * np.outer(v, v @ a[j:, j:])",
                         "a[j:, j:] -= 1.0 * np.outer(v, v @ a[j:, j:])"),
    # L of the LQ sweep not absorbed into the left neighbour (dropped term)
    "drop_L_absorb": ("G[k - 1] = np.tensordot(G[k - 1], l_mat, axes=([2], [0]))",
                      "G[k - 1] = G[k - 1]"),
    # R propagated transposed (wrong operand)
    "R_transposed": ("G[k + 1] = np.tensordot(r_mat, G[k + 1], axes=([1], [0]))",
                     "G[k + 1] = np.tensordot(r_mat.T, G[k + 1], axes=([1], [0]))"),
    # norm of g_n not absorbed into G_{n-1}
    "drop_norm_absorb": ("G[m - 1] = rho * G[m - 1]", "G[m - 1] = G[m - 1]"),
    # wrong sign in the temporal row
    "g_sign": ("self.g = a_mat.T @ x.reshape(-1)", "self.g = -(a_mat.T @ x.reshape(-1))"),
    # right interface built from the wrong core index
    "B_wrong_core": ("B[k] = np.tensordot(G[k + 1], B[k + 1], axes=([2], [0]))",
                     "B[k] = np.tensordot(G[min(k + 2, m - 1)], B[k + 1], axes=([2], [0]))"),
    # local solve contracted with B_k instead of B_k^T on the wrong axis order
    "local_solve_transpose": ("gt = np.tensordot(t_k, B[k].T, axes=([2], [0]))",
                              "gt = np.tensordot(t_k[:, ::-1, :], B[k].T, axes=([2], [0]))"),
    # global objective (all slices seen so far) summed over the current slice only; only the
    # all-slices pin exercises it
    "global_objective_current_only": ("    for i, x in enumerate(slices):",
                                      "    for i, x in enumerate(slices[-1:]):"),
    # stored cores contracted with the slice index and the right rank swapped (wrong index
    # order of the materialised left interface); only the all-slices pin exercises it
    "left_interface_index_order": ("a = (a @ c.reshape(r0, ik * r1)).reshape(-1, r1)",
                                   "a = (a @ c.transpose(0, 2, 1).reshape(r0, ik * r1)).reshape(-1, r1)"),
}

PINS = [
    "test_householder_rank_deficient_and_zero",
    "test_lq",
    "test_closed_form_subspace_iteration_n3",
    "test_closed_form_saturated_n4",
    "test_exact_recovery_noiseless_tt_stream",
    "test_monotonicity_prop41",
    "test_local_solve_is_bruteforce_least_squares",
    "test_temporal_row_is_bruteforce_lstsq",
    "test_all_slices_batch_least_squares",
]


def _mutant(name):
    src = open(ORACLE_SRC).read()
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    mod = types.ModuleType(f"ttals_oracle_mut_{name}")
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), mod.__dict__)
    return mod


def _run_pin(pins_mod, pin):
    import inspect
    fn = getattr(pins_mod, pin)
    params = list(inspect.signature(fn).parameters)
    marks = getattr(fn, "pytestmark", [])
    cases = [()]
    for mk in marks:
        if mk.name == "parametrize":
            cases = [c if isinstance(c, tuple) else (c,) for c in mk.args[1]]
    for case in cases:
        fn(*case) if params else fn()


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutation_is_caught(name):
    sys.path.insert(0, HERE)
    import test_oracle_pins as P
    original = P.O
    P.O = _mutant(name)
    caught = []
    try:
        for pin in PINS:
            try:
                _run_pin(P, pin)
            except Exception:          # AssertionError, or a shape error the mistake causes
                caught.append(pin)
    finally:
        P.O = original
    assert caught, f"mutation {name} passed every pin"


def test_unmutated_copy_passes_every_pin():
    """Control: the harness itself reports no failure for an unedited copy."""
    sys.path.insert(0, HERE)
    import test_oracle_pins as P
    original = P.O
    mod = types.ModuleType("ttals_oracle_copy")
    exec(compile(open(ORACLE_SRC).read(), "<copy>", "exec"), mod.__dict__)
    P.O = mod
    try:
        for pin in PINS:
            _run_pin(P, pin)
    finally:
        P.O = original
