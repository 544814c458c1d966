"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a fresh copy of an oracle module (a dropped
term, a flipped sign, a wrong index, a transposed operand, a wrong weight),
puts the copy in place of the module for the duration of the test, and runs
the pin that should notice it: the pin must fail.  The mistakes are planted
on the CPU, in the oracle only; nothing here touches the library.
"""
import os
import sys
import types

import pytest

import test_oracle_cpbc
import test_oracle_cpbc_minus
import test_oracle_dp5
import test_oracle_frame
import test_oracle_pins
import test_oracle_tensor_filter

PIN_MODULES = {"pins": test_oracle_pins, "cpbc": test_oracle_cpbc, "cpbc_minus": test_oracle_cpbc_minus,
               "dp5": test_oracle_dp5,
               "frame": test_oracle_frame, "tensor_filter": test_oracle_tensor_filter}

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _install_mutant(monkeypatch, modname, old, new):
    """Replace oracle.<modname> everywhere it is referenced (the package, the
    other oracle modules, the pin modules) by a copy whose source has the one
    occurrence of `old` replaced by `new`."""
    path = os.path.join(ROOT, "oracle", modname + ".py")
    with open(path) as f:
        src = f.read()
    assert src.count(old) == 1, "the planted mistake must match exactly one place: %r" % old
    full = "oracle." + modname
    orig = sys.modules[full]
    mod = types.ModuleType(full)
    mod.__file__ = path
    mod.__package__ = "oracle"
    exec(compile(src.replace(old, new), path, "exec"), mod.__dict__)
    monkeypatch.setitem(sys.modules, full, mod)
    for name, m in list(sys.modules.items()):
        if m is None or not (name == "oracle" or name.startswith("oracle.") or "test_oracle_" in name):
            continue
        for k, v in list(vars(m).items()):
            if v is orig:
                monkeypatch.setattr(m, k, mod)
    return mod


# (module, original text, planted mistake, pin, pin arguments)
CASES = {
    # GH right-hand side (oracle/gh.py)
    "T3 term sign": ("gh", '- np.einsum("...cd,...ef,...ace,...bdf->...ab", psi_inv, psi_inv, Gam, Gam))',
                     '+ np.einsum("...cd,...ef,...ace,...bdf->...ab", psi_inv, psi_inv, Gam, Gam))',
                     "test_rhs_of_exact_kerr_schild_converges_exponentially", (0.9, (3.0, 6.0))),
    # (psi^cd Pi_ca Pi_db vanishes on stationary Kerr-Schild data: only the
    # moving-coordinates flat-space pin sees this term)
    "Pi-Pi term sign": ("gh", '- np.einsum("...cd,...ca,...db->...ab", psi_inv, Pi, Pi)',
                        '+ np.einsum("...cd,...ca,...db->...ab", psi_inv, Pi, Pi)',
                        "test_rhs_equals_the_time_derivative_of_flat_space_in_moving_coordinates", ()),
    "t t Pi Pi term sign": ("gh", "- 0.5 * Nb * tPt[..., None, None] * Pi", "+ 0.5 * Nb * tPt[..., None, None] * Pi",
                            "test_rhs_equals_the_time_derivative_of_flat_space_in_moving_coordinates", ()),
    "dropped t.Pi g Phi term": ("gh", '- Nb * np.einsum("...i,...ij,...jab->...ab", tPi_i, ginv, Phi)\n', '\n',
                                "test_rhs_of_exact_kerr_schild_converges_exponentially", (0.9, (3.0, 6.0))),
    "Christoffel index": ("gh", 'Gam = 0.5 * (np.einsum("...bac->...abc", d)',
                          'Gam = 0.5 * (np.einsum("...cba->...abc", d)',
                          "test_rhs_equals_the_time_derivative_of_flat_space_in_moving_coordinates", ()),
    "nabla H without the Gamma term": ("gh", 'nablaH = dH4 - np.einsum("...cab,...c->...ab", Gam_up, H)',
                                       'nablaH = dH4 + 0.0 * np.einsum("...cab,...c->...ab", Gam_up, H)',
                                       "test_rhs_equals_the_time_derivative_of_flat_space_in_moving_coordinates", ()),
    "Phi equation t t Phi Pi term sign": ("gh", "+ 0.5 * Ni * np.einsum(\"...i,...ab->...iab\", tPhit, Pi)",
                                          "- 0.5 * Ni * np.einsum(\"...i,...ab->...iab\", tPhit, Pi)",
                                          "test_rhs_equals_the_time_derivative_of_flat_space_in_moving_coordinates", ()),
    "dropped gamma2 damping of Phi": ("gh", "              - gamma2 * Ni * Phi)", "              )",
                                      "test_three_index_constraint_decays_at_rate_gamma2_on_minkowski", ()),
    "gamma0 damping sign": ("gh", "+ gamma0 * Nb * damp", "- gamma0 * Nb * damp",
                            "test_gauge_constraint_damping_rates_on_minkowski", ()),
    "gamma2 sign in u^pm": ("gh", "wp = Pi + nPhi - gamma2 * psi", "wp = Pi + nPhi + gamma2 * psi",
                            "test_characteristic_round_trip", ()),
    "interface upwind sides swapped": ("gh", "new_i = np.where(neg, wo[q], wi[q])", "new_i = np.where(pos, wo[q], wi[q])",
                                       "test_interface_exchange_is_upwind_per_characteristic_family", (-1.0,)),
    "outer BC freezes outgoing": ("gh", "        mask = (v < 0.0)\n", "        mask = (v > 0.0)\n",
                                  "test_outer_bc_zeroes_only_incoming_fields", ()),
    "three-index constraint sign": ("gh", "    C3 = dpsi - Phi\n    C4 = np.einsum(", "    C3 = Phi - dpsi\n    C4 = np.einsum(",
                                    "test_constraint_components_of_fields_with_a_known_violation", ()),
    "four-index constraint antisymmetrised the wrong way": (
        "gh", 'C4 = np.einsum("...ijab->...ijab", dPhi) - np.einsum("...jiab->...ijab", dPhi)',
        'C4 = np.einsum("...jiab->...ijab", dPhi) - np.einsum("...ijab->...ijab", dPhi)',
        "test_constraint_components_of_fields_with_a_known_violation", ()),
    "interface results written to the wrong sides": (
        "evolve", "        out[s][nr - 1] = np.moveaxis(na, -1, 0)\n        out[s + 1][0] = np.moveaxis(nb, -1, 0)",
        "        out[s][nr - 1] = np.moveaxis(nb, -1, 0)\n        out[s + 1][0] = np.moveaxis(na, -1, 0)",
        "test_domain_boundaries_touch_only_boundary_slices_and_upwind_by_side", ()),
    "inverse spacetime metric sign": (
        "gh", 'psi_inv[..., 1:, 1:] = ginv - np.einsum("...i,...j->...ij", beta_up, beta_up)',
        'psi_inv[..., 1:, 1:] = ginv + np.einsum("...i,...j->...ij", beta_up, beta_up)',
        "test_inverse_spacetime_metric", ()),
    "boundary normal not raised": ("gh", 'n_up = np.einsum("...ij,...j->...i", s["ginv"], n_dn)', "n_up = n_dn",
                                   "test_characteristic_round_trip", ()),
    # grid coordinates (oracle/grid.py)
    "x and y swapped in the coordinates": ("grid", "    X = r * st * cp\n    Y = r * st * sp\n",
                                           "    X = r * st * sp\n    Y = r * st * cp\n",
                                           "test_cartesian_gradient_exact_on_polynomials", (9, 5, 5)),
    # spectral maps (oracle/spectral.py)
    "Chebyshev derivative recurrence": ("spectral", "b[k] = (b[k + 2] + 2.0 * (k + 1) * a[k + 1]) / cb",
                                        "b[k] = (b[k + 2] + 2.0 * k * a[k + 1]) / cb",
                                        "test_radial_derivative_exact_below_degree_n_r", ()),
    "Y_lm normalisation": ("spectral", "        return np.sqrt(2.0) * np.cos(m * phi)\n",
                           "        return np.cos(m * phi)\n", "test_real_ylm_and_dtheta_match_scipy", (7,)),
    "DiffJac entry sign": ("spectral", "J[2, 1] = -st / r * one", "J[2, 1] = st / r * one",
                           "test_cartesian_gradient_exact_on_polynomials", (9, 5, 5)),
    "DiffJac transposed": ("spectral", "J[1, 0] = st * sp * one\n    J[2, 0] = ct * one\n    J[0, 1] = ct * cp / r * one",
                           "J[1, 0] = ct * cp / r * one\n    J[2, 0] = ct * one\n    J[0, 1] = st * sp * one",
                           "test_cartesian_gradient_exact_on_polynomials", (9, 5, 5)),
    "ExpCheb exponent": ("spectral", "return np.exp(-alpha * (k / (n - 1.0)) ** order)",
                         "return np.exp(-alpha * (k / (n - 1.0)) ** (2 * order))",
                         "test_expcheb_filter_scales_each_chebyshev_mode", ()),
    "d/dphi harmonic sign": ("spectral", "        return -np.sqrt(2.0) * m * np.sin(m * phi)\n",
                             "        return np.sqrt(2.0) * m * np.sin(m * phi)\n",
                             "test_cartesian_gradient_exact_on_polynomials", (9, 5, 5)),
    "SH truncation keeps one l too few": ("spectral", "mask = np.array([1.0 if l <= keep_l else 0.0",
                                          "mask = np.array([1.0 if l < keep_l else 0.0",
                                          "test_sh_truncation_filter_keeps_low_l_and_drops_high_l", ()),
    # perturbations (oracle/perturb.py)
    "pulse Phi without the radial factor": ("perturb", "    fr = A * dG * S[None]\n", "    fr = A * G * S[None]\n",
                                            "test_psi_pulse_phi_is_the_gradient_of_psi", ()),
    "pulse moving outward": ("perturb", "pi = -(fr - bdf) / s[\"alpha\"]", "pi = (fr - bdf) / s[\"alpha\"]",
                             "test_psi_pulse_is_ingoing_on_flat_space", ()),
    "Chebyshev analysis end weight": ("spectral", "cbar[0] = cbar[-1] = 2.0\n    a = np.zeros_like(u, dtype=float)",
                                      "cbar[0] = 2.0\n    a = np.zeros_like(u, dtype=float)",
                                      "test_radial_derivative_exact_below_degree_n_r", ()),
    "harmonic analysis without the theta weights": ("spectral", 'w = g["wth"][:, None] * g["wphi"]',
                                                    'w = 0.5 + 0.0 * g["wth"][:, None] * g["wphi"]',
                                                    "test_sh_truncation_filter_keeps_low_l_and_drops_high_l", ()),
    "Pi modes with the Gaussian's width squared twice": (
        "perturb", "    G = np.exp(-((r - Rc) / w) ** 2)\n    du = np.zeros(",
        "    G = np.exp(-((r - Rc) / w) ** 4)\n    du = np.zeros(",
        "test_pi_modes_recover_their_coefficients", ()),
    # Kerr-Schild data, spin-vector form (oracle/kerr_schild.py)
    "spin-vector Kerr-Schild rotating the wrong way": (
        "kerr_schild", "(r * X[i] - cross[i] + ad * A[i] / r)", "(r * X[i] + cross[i] + ad * A[i] / r)",
        "test_spin_vector_along_z_matches_the_scalar_form", ()),
    # quadrature (oracle/grid.py)
    "volume element without r^2": ("grid", "wr = g[\"wr\"] * 0.5 * (g[\"r_out\"] - g[\"r_in\"]) * g[\"r\"] ** 2",
                                   "wr = g[\"wr\"] * 0.5 * (g[\"r_out\"] - g[\"r_in\"]) * g[\"r\"]",
                                   "test_volume_weights_sum_to_shell_volume", ()),
    "Clenshaw-Curtis end weights": ("grid", "c = 1.0 if j in (0, N) else 2.0", "c = 2.0 if j in (0, N) else 1.0",
                                    "test_clenshaw_curtis_exact_on_polynomials", (11,)),
    # time stepper (oracle/evolve.py)
    "RK4 weights": ("evolve", "dt / 6.0 * (p + 2.0 * q + 2.0 * r + s)", "dt / 6.0 * (p + 2.0 * q + r + 2.0 * s)",
                    "test_rk4_matches_stability_polynomial", "monkeypatch"),
    "RK4 second stage node": ("evolve", "k2 = rhs(dom, [a + 0.5 * dt * k for a, k in zip(u, k1)])",
                              "k2 = rhs(dom, [a + dt * k for a, k in zip(u, k1)])",
                              "test_rk4_matches_stability_polynomial", "monkeypatch"),
    # Kerr-Schild data (oracle/kerr_schild.py)
    "Kerr-Schild H": ("kerr_schild", "H = M * r ** 3 / (r ** 4 + a * a * z * z)",
                      "H = M * r ** 3 / (r ** 4 - a * a * z * z)",
                      "test_rhs_of_exact_kerr_schild_converges_exponentially", (0.9, (3.0, 6.0))),
    # tensor spherical-harmonic filter (oracle/tensor_filter.py)
    "tensor filter back-projection without conjugate": (
        "tensor_filter", "w = w * np.conj(E[A[k]][I[k]])", "w = w * E[A[k]][I[k]]",
        "tensor_filter::test_idempotent_and_real_on_random_fields", ()),
    "spin weights of the frame vectors": (
        "tensor_filter", "np.conj(m)]), [0, 1, -1]", "np.conj(m)]), [0, -1, 1]",
        "tensor_filter::test_vector_harmonics_pass_below_and_vanish_above_the_cut", (2, 1)),
    # Dormand-Prince pair (oracle/dp5.py)
    "DP5 stage coefficient": ("dp5", "[_F(44, 45), _F(-56, 15), _F(32, 9)],", "[_F(44, 45), _F(-56, 15), _F(32, 7)],",
                              "dp5::test_fifth_order_weights_satisfy_all_order_conditions_exactly", ()),
    "DP5 embedded weight": ("dp5", "_F(187, 2100)", "_F(187, 2000)",
                            "dp5::test_fourth_order_companion_is_order_four_not_five", ()),
    "DP5 controller exponent": ("dp5", "SAFETY * err ** (-0.2)", "SAFETY * err ** (-0.25)",
                                "dp5::test_controller_rejects_large_steps_and_clamps_growth", ()),
    "DP5 error estimate without dt": ("dp5", "e = [dt * sum((b[j] - bh[j]) * k[j][i]", "e = [sum((b[j] - bh[j]) * k[j][i]",
                                      "dp5::test_observed_orders_of_solution_and_error_estimate", ()),
    "spin-weighted harmonic phase": ("tensor_filter", "pref = (-1) ** m * sqrt(", "pref = sqrt(",
                                     "tensor_filter::test_spin_zero_is_scipy_ylm_and_eth_raises_spin", ()),
    # rotating frame (oracle/frame.py)
    "grid velocity sign": ("frame", "xdot = omega * np.cross(", "xdot = -omega * np.cross(",
                           "frame::test_rotating_exact_solution_matches_its_time_derivative",
                           [(1.0, 0.0, (0.3, -0.5, 0.8)), (1.0, 0.7, (0.0, 0.0, 1.0))]),
    "rotated Phi with the transposed rotation": (
        "frame", 'Phi2 = np.einsum("ij,ac,bd,...jcd->...iab", R, L, L, Phi)',
        'Phi2 = np.einsum("ji,ac,bd,...jcd->...iab", R, L, L, Phi)',
        "frame::test_rotating_exact_solution_matches_its_time_derivative",
        [(1.0, 0.0, (0.3, -0.5, 0.8)), (1.0, 0.7, (0.0, 0.0, 1.0))]),
    "rotated gauge derivative with the transposed rotation": (
        "frame", 'np.einsum("ij,ab,...jb->...ia", R, L, dH)', 'np.einsum("ji,ab,...jb->...ia", R, L, dH)',
        "frame::test_rotating_exact_solution_matches_its_time_derivative",
        [(1.0, 0.0, (0.3, -0.5, 0.8)), (1.0, 0.7, (0.0, 0.0, 1.0))]),
    # time-integrated constraint energy (oracle/evolve.py, R13)
    "constraint energy summed from the initial state": (
        "evolve", "u = rk4_step(dom, u, dt)\n        _, norms = constraints(dom, u)",
        "_, norms = constraints(dom, u)\n        u = rk4_step(dom, u, dt)",
        "test_constraint_energy_sums_the_rk4_decay_of_a_violation_on_flat_space", ()),
    "constraint energy without the step size": (
        "evolve", "E += dt * sum(norms)", "E += sum(norms)",
        "test_constraint_energy_sums_the_rk4_decay_of_a_violation_on_flat_space", ()),
    # general time-dependent map (oracle/frame.py, oracle/gh.py)
    "moving frame without the expansion's Jacobian": (
        "frame", 'dUi = np.einsum("kj,...jf->...kf", R, dUg) / a', 'dUi = np.einsum("kj,...jf->...kf", R, dUg)',
        "frame::test_moving_exact_solution_matches_its_time_derivative_under_a_general_map",
        [("contraction+translation",), ("expand+translate+tilted rotation",)]),
    "moving boundary speed shift with the wrong sign": (
        "gh", 'sh = bg.get("n_xdot", 0.0)', 'sh = -bg.get("n_xdot", 0.0)',
        "frame::test_a_boundary_outrunning_every_family_freezes_them_all", ()),
    "moving boundary normal from the fixed centre": (
        "frame", "xc = x[ir] - T", "xc = x[ir]",
        "frame::test_translated_boundary_normal_points_from_the_moving_centre", ()),
    # constraint-preserving outer condition (oracle/gh.py)
    "constraint-preserving correction sign": (
        "gh", "wpsi = np.where(inc_psi, wpsi + v_psi[..., None, None] * nC3, wpsi)",
        "wpsi = np.where(inc_psi, wpsi - v_psi[..., None, None] * nC3, wpsi)",
        "cpbc::test_constraint_preserving_upsi_removes_the_normal_derivative", ()),
    # the u^- constraint part of the outer condition (oracle/gh.py)
    "gauge constraint derivative without the inverse-metric variation": (
        "gh", 'return (w + np.einsum("...bc,...abc->...a", dpsi_inv, Gam)',
        'return (w + 0.0 * np.einsum("...bc,...abc->...a", dpsi_inv, Gam)',
        "cpbc_minus::test_gauge_constraint_derivative_matches_central_differences", ()),
    "gauge constraint derivative with the lapse variation doubled": (
        "gh", "dN = 0.5 * N ** 3 * dpsi_inv[..., 0, 0]", "dN = N ** 3 * dpsi_inv[..., 0, 0]",
        "cpbc_minus::test_gauge_constraint_derivative_matches_central_differences", ()),
    "incoming constraint field with the shift term's sign flipped": (
        "gh", 'return ((dtC - np.einsum("...i,...ia->...a", beta, dC))',
        'return ((dtC + np.einsum("...i,...ia->...a", beta, dC))',
        "cpbc_minus::test_uminus_condition_ignores_the_normal_derivative_of_uminus", ()),
    "Bjorhus weight with the shift term's sign flipped": (
        "gh", "((N - nb) / (2.0 * N))", "((N + nb) / (2.0 * N))",
        "cpbc_minus::test_uminus_condition_ignores_the_normal_derivative_of_uminus", ()),
    "u^- condition along the corrected time derivative (no Bjorhus weight)": (
        "gh", "target = -K(dudt0) + ((N - nb) / (2.0 * N))[..., None] * K(dudt_int)",
        "target = -K(dudt0) + 0.0 * K(dudt_int)",
        "cpbc_minus::test_uminus_condition_ignores_the_normal_derivative_of_uminus", ()),
    "incoming constraint field along the incoming null direction": (
        "gh", """                + np.einsum("...i,...ia->...a", n_up, dC))""",
        """                - np.einsum("...i,...ia->...a", n_up, dC))""",
        "cpbc_minus::test_uminus_condition_ignores_the_normal_derivative_of_uminus", ()),
    "u^- subspace condition on k instead of l": (
        "gh", 'M[..., 4, 0:4] = tet["l_up"]', 'M[..., 4, 0:4] = tet["k_up"]',
        "cpbc_minus::test_uminus_derivative_lies_in_the_constraint_subspace", ()),
    "transverse projector without the t t term": (
        "gh", 'P = psi4 + np.einsum("...a,...b->...ab", t_dn, t_dn) - np.einsum',
        'P = psi4 - np.einsum',
        "cpbc_minus::test_uminus_derivative_lies_in_the_constraint_subspace", ()),
}


def _fails(fn, args):
    try:
        fn(*args)
    except AssertionError:
        return True
    return False


@pytest.mark.parametrize("name", sorted(CASES))
def test_pin_catches_planted_mistake(name, monkeypatch):
    """The pin passes on the real oracle (for every argument set) and fails on
    the planted mistake (for at least one)."""
    modname, old, new, pin, args = CASES[name]
    where, _, fname = pin.rpartition("::")
    pin_fn = getattr(PIN_MODULES[where or "pins"], fname)
    if args == "monkeypatch":
        arg_sets = [(monkeypatch,)]
    else:
        arg_sets = args if isinstance(args, list) else [args]
    for a in arg_sets:
        pin_fn(*a)
    _install_mutant(monkeypatch, modname, old, new)
    assert any(_fails(pin_fn, a) for a in arg_sets), "no pin failed on: " + name
