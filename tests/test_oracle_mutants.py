"""The oracle's pins catch plausible mistakes (CPU only).

Each case plants one mistake in a copy of oracle/lbm_oracle.c: a dropped
term, a wrong sign, index or constant, a transposed operand, a missing
factor.  The copy is compiled into a library of its own, the oracle's
Python wrappers are pointed at it, and the pins named for the case run
against it: at least one of them must fail.  The real oracle passes all of
them (tests/test_oracle_pins.py).
"""
import ctypes as C
import os
import subprocess

import numpy as np
import pytest

import oracle
import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "lbm_oracle.c")
G0, G1 = (1.0, 1.0, 1.0, 1.0), (0.8, 1.2, 1.5, 0.5)

# name: (mistake, text in the oracle, planted text, pins expected to catch it)
MUTANTS = {
    "one_d_weight": (
        "1-D weight of c = +-1 mistyped (Appendix A)",
        "? 2.0 / 3.0 : 1.0 / 6.0", "? 2.0 / 3.0 : 1.0 / 5.0",
        [("test_weights_quadrature_moments",), ("test_central_equilibrium_moments_vanish", 0)]),
    "hermite_cyc_sign": (
        "wrong sign of the delta terms of the Hermite polynomials (Appendix A)",
        "r -= ORC_THETA0 * orc_hermite(rest, n - 2, xi);", "r += ORC_THETA0 * orc_hermite(rest, n - 2, xi);",
        [("test_hermite_matches_printed_forms",), ("test_central_equilibrium_moments_vanish", 0)]),
    "equilibrium_second_order_only": (
        "equilibrium truncated at second order instead of the full expansion (Appendix A)",
        "g_eq_prefactor[m] = mult / (factorial(n) * pow(ORC_THETA0, n));",
        "g_eq_prefactor[m] = n > 2 ? 0.0 : mult / (factorial(n) * pow(ORC_THETA0, n));",
        [("test_central_equilibrium_moments_vanish", 0), ("test_equilibrium_closed_forms", 0)]),
    "equilibrium_multiplicity": (
        "index tuples of one multi-index counted once (Sec. 2.1 equilibrium sum)",
        "double mult = factorial(n) / (factorial(deg[0]) * factorial(deg[1]) * factorial(deg[2]));",
        "double mult = 1.0;",
        [("test_equilibrium_closed_forms", 0), ("test_central_equilibrium_moments_vanish", 0)]),
    "central_shift_sign": (
        "moments taken about c + u instead of c - u (Sec. 2.1 central moments)",
        "double xi[3] = {c[0] - u[0], c[1] - u[1], c[2] - u[2]};",
        "double xi[3] = {c[0] + u[0], c[1] + u[1], c[2] + u[2]};",
        [("test_central_equilibrium_moments_vanish", 0), ("test_collision_relaxes_each_central_moment", G0)]),
    "off_diagonal_rate": (
        "off-diagonal second-order moments relaxed at 1 instead of omega (Appendix A)",
        "    if (n == 2) return omega;", "    if (n == 2) return (m == 2 || m == 6 || m == 18) ? omega : 1.0;",
        [("test_collision_reduces_to_bgk", 0.6), ("test_collision_relaxes_each_central_moment", G0)]),
    "ghost_rate_order": (
        "ghost rates assigned to the wrong orders",
        "    return ghost[n - 3];", "    return ghost[6 - n];",
        [("test_collision_relaxes_each_central_moment", G1)]),
    "momentum_for_velocity": (
        "rho u used where u is meant",
        "mom[1 + a] = j[a] / rho;", "mom[1 + a] = j[a];",
        [("test_collision_conserves_mass_momentum", 0)]),
    "solve_rhs_not_swapped": (
        "pivoting swaps the rows of the matrix but not of the right-hand side",
        "            double t = b[k]; b[k] = b[p]; b[p] = t;", "            (void)0;",
        [("test_gaussian_elimination_matches_lapack",), ("test_collision_conserves_mass_momentum", 1)]),
    "push_for_pull": (
        "streaming gathers from x + c_i instead of x - c_i",
        "int fl = flag_at(L, x - c[0], y - c[1], z - c[2], &src);",
        "int fl = flag_at(L, x + c[0], y + c[1], z + c[2], &src);",
        [("test_streaming_pull_and_bounce_back", 0), ("test_viscous_stress_shear_wave",)]),
    "bounce_back_same_direction": (
        "a wall link returns population i instead of its opposite (Sec. 2.2 bounce-back)",
        "const int ib = ORC_Q - 1 - i;", "const int ib = i;",
        [("test_closed_box_conserves_mass",), ("test_streaming_pull_and_bounce_back", 0)]),
    "bouzidi_near_weights_swapped": (
        "the two weights of Bouzidi's q < 1/2 interpolation exchanged",
        "fi = 2.0 * q * fin[self * ORC_Q + ib] + (1.0 - 2.0 * q) * fin[nbr * ORC_Q + ib];",
        "fi = (1.0 - 2.0 * q) * fin[self * ORC_Q + ib] + 2.0 * q * fin[nbr * ORC_Q + ib];",
        [("test_interpolated_bounce_back_places_the_walls",)]),
    "bouzidi_far_wrong_population": (
        "Bouzidi's q >= 1/2 form mixes with f_ib instead of f_i",
        "fi = fin[self * ORC_Q + ib] / (2.0 * q) + (1.0 - 1.0 / (2.0 * q)) * fin[self * ORC_Q + i];",
        "fi = fin[self * ORC_Q + ib] / (2.0 * q) + (1.0 - 1.0 / (2.0 * q)) * fin[self * ORC_Q + ib];",
        [("test_interpolated_bounce_back_places_the_walls",)]),
    "nee_sign": (
        "non-equilibrium part subtracted instead of added (Sec. 2.2 NEE)",
        "fout[b * ORC_Q + i] = feq_b[i] + (fout[bf * ORC_Q + i] - feq_f[i]);",
        "fout[b * ORC_Q + i] = feq_b[i] - (fout[bf * ORC_Q + i] - feq_f[i]);",
        [("test_nee_boundary_nodes",)]),
    "outlet_density": (
        "outlet takes the partner's density instead of the imposed one",
        "rho_b = L->rho_out;", "rho_b = rho_f;",
        [("test_nee_boundary_nodes",)]),
    "inlet_density": (
        "inlet density fixed at 1 instead of extrapolated",
        "            rho_b = rho_f;\n            orc_inlet_velocity", "            rho_b = 1.0;\n            orc_inlet_velocity",
        [("test_nee_boundary_nodes",)]),
    "parabola": (
        "parabolic inlet profile with 2 r^2 instead of 4 r^2 (Sec. 2.2 inlet profile)",
        "(1.0 - 4.0 * r2 / (L->d_in * L->d_in))", "(1.0 - 2.0 * r2 / (L->d_in * L->d_in))",
        [("test_nee_boundary_nodes",)]),
    "ramp_shape": (
        "start-up ramp s^2 instead of s^2 (3 - 2 s)",
        "double r = s * s * (3.0 - 2.0 * s);", "double r = s * s;",
        [("test_inlet_start_up_ramp",)]),
    "noise_bits": (
        "noise keeps 23 bits instead of 24",
        "(double)(h >> 40) * (1.0 / 8388608.0) - 1.0", "(double)(h >> 41) * (1.0 / 8388608.0) - 1.0",
        [("test_noise_uniform",)]),
    "splitmix_constant": (
        "a SplitMix64 multiplier mistyped",
        "z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;", "z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b8ULL;",
        [("test_splitmix64_reference_outputs",)]),
    "noise_ignores_seed": (
        "the seed's hash dropped from the noise counter chain",
        "h = orc_splitmix64((uint64_t)step + h);", "h = orc_splitmix64((uint64_t)step);",
        [("test_noise_depends_on_every_counter",)]),
    "stress_sign": (
        "strain rate without the minus sign (Appendix A strain-rate relation)",
        "const double S = -a / (2.0 * rho * ORC_THETA0 * tau);", "const double S = a / (2.0 * rho * ORC_THETA0 * tau);",
        [("test_viscous_stress_shear_wave",)]),
    "stress_theta_term": (
        "theta0 delta_ab left out of the second-order Hermite moment",
        "            if (pa[k] == pb[k]) h -= ORC_THETA0;", "            if (pa[k] == pb[k]) h -= 0.0;",
        [("test_viscous_stress_of_equilibrium_is_zero",)]),
    "node_stress_dropped": (
        "inlet/outlet nodes report no stress instead of their partner's",
        "for (int k = 0; k < 6; ++k) sigma[b * 6 + k] = sigma[bf * 6 + k];",
        "for (int k = 0; k < 6; ++k) sigma[b * 6 + k] = 0.0;",
        [("test_square_duct_poiseuille_profile",)]),
    "inlet_axis_offset": (
        "radius measured from the cell corner instead of its centre",
        "double rx = x + 0.5 - L->axis_x, ry = y + 0.5 - L->axis_y;", "double rx = x - L->axis_x, ry = y - L->axis_y;",
        [("test_nee_boundary_nodes",)]),
    "parabola_peak": (
        "parabolic profile peaking at u0 instead of 2 u0 (Sec. 2.2 inlet profile)",
        "speed = 2.0 * L->u_in * (1.0 - 4.0 * r2", "speed = L->u_in * (1.0 - 4.0 * r2",
        [("test_nee_boundary_nodes",)]),
    "noise_not_scaled_by_u0": (
        "inlet perturbation not scaled by the mean inlet velocity",
        "u[a] += L->noise_amp * L->u_in * orc_noise(L->seed, step, node, a);",
        "u[a] += L->noise_amp * orc_noise(L->seed, step, node, a);",
        [("test_nee_boundary_nodes",)]),
    "noise_counter_packing": (
        "node and component packed so that two pairs share a counter",
        "h = orc_splitmix64((((uint64_t)node << 2) | (uint64_t)comp) + h);",
        "h = orc_splitmix64((((uint64_t)node << 1) + (uint64_t)comp) + h);",
        [("test_noise_depends_on_every_counter",)]),
    "outlet_velocity_zero": (
        "outlet velocity set to zero instead of extrapolated",
        "for (int a = 0; a < 3; ++a) u_b[a] = u_f[a];", "for (int a = 0; a < 3; ++a) u_b[a] = 0.0;",
        [("test_nee_boundary_nodes",), ("test_plug_flow_is_fixed_point",)]),
    "inlet_direction": (
        "inlet speed put on every axis instead of along the inward normal",
        "u[a] = speed * n[a];", "u[a] = speed;",
        [("test_nee_boundary_nodes",)]),
    "nee_previous_partner": (
        "NEE takes the partner's populations of the previous step",
        "fout[b * ORC_Q + i] = feq_b[i] + (fout[bf * ORC_Q + i] - feq_f[i]);",
        "fout[b * ORC_Q + i] = feq_b[i] + (fin[bf * ORC_Q + i] - feq_f[i]);",
        [("test_nee_boundary_nodes",)]),
    "nee_partner_not_unique": (
        "a boundary node with several fluid axis neighbours accepted",
        "return count == 1 ? found : -1;", "return count >= 1 ? found : -1;",
        [("test_nee_partner_must_be_unique",)]),
    "stress_component_pairs": (
        "stress components xy and xz exchanged",
        "static const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 1, 2, 2};",
        "static const int pa[6] = {0, 1, 2, 0, 0, 1}, pb[6] = {0, 1, 2, 2, 1, 2};",
        [("test_viscous_stress_shear_wave",)]),
    "stress_viscosity": (
        "viscosity theta0 tau instead of theta0 (tau - 1/2)",
        "nu = ORC_THETA0 * (tau - 0.5);", "nu = ORC_THETA0 * tau;",
        [("test_viscous_stress_shear_wave",)]),
    "stress_from_post_collision": (
        "stress taken from the post-collision instead of the gathered populations",
        "        gather(L, fin, x, y, z, f);\n        orc_viscous_stress(f, L->omega, sigma + b * 6);",
        "        for (int i = 0; i < ORC_Q; ++i) f[i] = fin[b * ORC_Q + i];\n"
        "        orc_viscous_stress(f, L->omega, sigma + b * 6);",
        [("test_viscous_stress_shear_wave",)]),
    "wall_distance_scale": (
        "wall distances decoded in 1/255 instead of 1/256",
        "const double q = L->wall_q[self * ORC_Q + i] / 256.0;", "const double q = L->wall_q[self * ORC_Q + i] / 255.0;",
        [("test_interpolated_bounce_back_places_the_walls",)]),
    "bouzidi_near_branch_missing": (
        "the q < 1/2 branch of Bouzidi's interpolation never taken",
        "if (q < 0.5) {", "if (q < 0.0) {",
        [("test_interpolated_bounce_back_places_the_walls",)]),
    "back_substitution_sign": (
        "wrong sign in the back substitution",
        "for (int j = k + 1; j < n; ++j) s -= A[k * n + j] * b[j];", "for (int j = k + 1; j < n; ++j) s += A[k * n + j] * b[j];",
        [("test_gaussian_elimination_matches_lapack",)]),
    "equilibrium_axis": (
        "equilibrium coefficients built from u_x on every axis",
        "for (int k = 0; k < n; ++k) a[m] *= u[idx[k]];", "for (int k = 0; k < n; ++k) a[m] *= u[0];",
        [("test_equilibrium_closed_forms", 0)]),
    "momentum_axis": (
        "momentum summed with c_x on every axis",
        "for (int a = 0; a < 3; ++a) j[a] += c[a] * f[i];", "for (int a = 0; a < 3; ++a) j[a] += c[0] * f[i];",
        [("test_collision_conserves_mass_momentum", 0)]),
    "raw_instead_of_central": (
        "raw Hermite moments H_m(c) instead of central ones H_m(c - u)",
        "double xi[3] = {c[0] - u[0], c[1] - u[1], c[2] - u[2]};",
        "double xi[3] = {(double)c[0], (double)c[1], (double)c[2]};",
        [("test_central_equilibrium_moments_vanish", 0)]),
    "totals_momentum": (
        "total momentum summed without the velocities",
        "for (int a = 0; a < 3; ++a) v[1 + a] += c[a] * fi;", "for (int a = 0; a < 3; ++a) v[1 + a] += fi;",
        [("test_totals_compensated",)]),
    "hermite_pairs_any_index": (
        "Hermite delta terms paired across different axes",
        "        if (idx[k] != idx[0]) continue;\n", "        (void)0;\n",
        [("test_hermite_matches_printed_forms",), ("test_central_equilibrium_moments_vanish", 0)]),
    "moment_index_degrees": (
        "x and y degrees of the moment multi-index exchanged",
        "    deg[0] = m % 3;\n    deg[1] = (m / 3) % 3;", "    deg[1] = m % 3;\n    deg[0] = (m / 3) % 3;",
        [("test_central_equilibrium_moments_vanish", 0)]),
    "velocity_index": (
        "y and z components of the stencil velocity exchanged",
        "    c[1] = (i / 3) % 3 - 1;\n    c[2] = i / 9 - 1;", "    c[2] = (i / 3) % 3 - 1;\n    c[1] = i / 9 - 1;",
        [("test_central_equilibrium_moments_vanish", 0)]),
    "theta0_perturbed": (
        "stencil temperature off by 1e-9",
        "#define ORC_THETA0 (1.0 / 3.0)", "#define ORC_THETA0 (1.0 / 3.0 + 1e-9)",
        [("test_central_equilibrium_moments_vanish", 0)]),
    "relaxation_sign": (
        "relaxation applied away from equilibrium",
        "rhs[m] = rate_of(m, omega, ghost, omega_cons) * s;", "rhs[m] = -rate_of(m, omega, ghost, omega_cons) * s;",
        [("test_collision_reduces_to_bgk", 0.6)]),
    "relaxation_without_f": (
        "collision relaxes f^eq instead of f^eq - f",
        "for (int i = 0; i < ORC_Q; ++i) d[i] = feq[i] - f[i];", "for (int i = 0; i < ORC_Q; ++i) d[i] = feq[i];",
        [("test_collision_conserves_mass_momentum", 0)]),
    "closed_faces_wrap": (
        "non-periodic faces treated as periodic",
        "    return periodic ? 1 : 0;", "    return 1;",
        [("test_streaming_pull_and_bounce_back", 0), ("test_nee_partner_must_be_unique",)]),
    "ramp_starts_late": (
        "start-up ramp one step late",
        "double s = (double)step / (double)L->ramp;", "double s = (double)(step - 1) / (double)L->ramp;",
        [("test_inlet_start_up_ramp",)]),
    "node_moments_not_read_back": (
        "field readback leaves out the inlet/outlet nodes",
        "        if (L->flags[b] == ORC_SOLID) { for (int a = 0; a < 4; ++a) mom[b * 4 + a] = 0.0; continue; }",
        "        if (L->flags[b] != ORC_FLUID) { for (int a = 0; a < 4; ++a) mom[b * 4 + a] = 0.0; continue; }",
        [("test_nee_boundary_nodes",)]),
    "node_moments_recorded_wrong": (
        "the step records the partner's density at an inlet/outlet node",
        "        m[b * 4] = rho_b;", "        m[b * 4] = rho_f;",
        [("test_nee_boundary_nodes",)]),
    "totals_uncompensated": (
        "compensation dropped from the FP64 totals",
        "comp[k] = (t - s[k]) - y;", "comp[k] = 0.0;",
        [("test_totals_compensated_on_an_ill_conditioned_sum",)]),
}


@pytest.fixture(scope="module")
def mutant_dir(tmp_path_factory):
    return tmp_path_factory.mktemp("oracle_mutants")


def build_mutant(directory, name, old, new):
    text = open(SRC).read()
    assert text.count(old) == 1, "the oracle text of %s is no longer unique" % name
    src = os.path.join(str(directory), name + ".c")
    lib = os.path.join(str(directory), name + ".so")
    with open(src, "w") as fh:
        fh.write(text.replace(old, new))
    flags = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]
    r = subprocess.run(["gcc"] + flags + ["-fopenmp", src, "-o", lib, "-lm"], capture_output=True)
    if r.returncode != 0:  # OpenMP is optional, as for the oracle itself
        subprocess.run(["gcc"] + flags + [src, "-o", lib, "-lm"], check=True, capture_output=True)
    return lib


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(mutant_dir, name):
    what, old, new, catchers = MUTANTS[name]
    lib = build_mutant(mutant_dir, name, old, new)
    saved = oracle.lib()
    oracle._lib = oracle.declare(C.CDLL(lib))
    caught = []
    try:
        with np.errstate(all="ignore"):
            for pin, *args in catchers:
                try:
                    getattr(pins, pin)(oracle, *args)
                except (AssertionError, RuntimeError, ValueError, ArithmeticError, np.linalg.LinAlgError):
                    caught.append(pin)  # a failed check, or the broken oracle failing outright
    finally:
        oracle._lib = saved
    assert caught, "no pin caught: " + what


# Mistakes in the oracle's Python side: the per-step sampled time averages.
def _sampled_after_step(self, n):
    """step_sampled with the stress sampled after the step instead of before it."""
    pairs = [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)]
    acc = dict(u=np.zeros((self.ncell, 3)), uu=np.zeros((self.ncell, 6)), sigma=np.zeros((self.ncell, 6)),
               rho=np.zeros(self.ncell))
    for _ in range(n):
        self.step(1)
        acc["sigma"] += self.field_stress()
        m = self.last_moments
        acc["u"] += m[:, 1:4]
        acc["uu"] += np.stack([m[:, 1 + a] * m[:, 1 + b] for a, b in pairs], axis=1)
        acc["rho"] += m[:, 0]
    return {k: v / n for k, v in acc.items()}


def _sampled_one_too_many(self, n, _orig=oracle.Lattice.step_sampled):
    """step_sampled dividing the sums by n + 1."""
    return {k: v * n / (n + 1) for k, v in _orig(self, n).items()}


@pytest.mark.parametrize("broken", [_sampled_after_step, _sampled_one_too_many], ids=lambda f: f.__name__)
def test_pins_catch_planted_mistake_in_sampling(monkeypatch, broken):
    monkeypatch.setattr(oracle.Lattice, "step_sampled", broken)
    with pytest.raises(AssertionError):
        pins.test_sampled_time_averages_of_a_decaying_wave(oracle)
