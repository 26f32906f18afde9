"""The oracle's pins catch plausible mistakes.

Each case plants one mistake in a copy of the oracle source (CPU only), compiles it,
and runs the pins of test_oracle_pins against it: at least one pin must fail.  This is
the evidence that the pins constrain every term of the step, not just the happy path.
"""
import os

import pytest

import oracle
import test_oracle_pins as pins
import test_oracle_variants as variants

# (name, text in dem_oracle.c, replacement, pins expected to notice)
MUTANTS = [
    ("normal stiffness factor", "    kn = 4.0 / 3.0 * Ye * sq;", "    kn = 1.0 * Ye * sq;",
     ["test_static_overlap_on_plane_matches_hertz"]),
    ("Young mixing ignores the wall",
     "  double Yw = eff_young(&c->particle, &c->wall);", "  double Yw = eff_young(&c->particle, &c->particle);",
     ["test_static_overlap_on_plane_matches_hertz"]),
    ("effective mass of a pair", "double me = 1.0 / (1.0 / s->m[i] + 1.0 / s->m[j]);",
     "double me = s->m[i];", [("test_restitution_recovers_input_coefficient", dict(e=0.7, v_rel=1.0))]),
    ("effective radius of a pair", "double Re = 1.0 / (1.0 / s->R[i] + 1.0 / s->R[j]);",
     "double Re = s->R[i];", ["test_hertz_head_on_contact_time_and_depth"]),
    ("normal damping factor", "    eta_n = -2.0 * sqrt(5.0 / 6.0) * beta * sqrt(Sn * me);",
     "    eta_n = -2.0 * beta * sqrt(Sn * me);", ["test_restitution_on_wall"]),
    ("beta without pi", "return le / sqrt(le * le + ORC_PI * ORC_PI);", "return le / sqrt(le * le + 1.0);",
     ["test_restitution_on_wall"]),
    ("tangential stiffness factor", "    kt = 8.0 * Ge * sq;", "    kt = 4.0 * Ge * sq;",
     ["test_tangential_stiffness_mindlin_with_rolling_coupling"]),
    ("shear-modulus mixing", "return 1.0 / (2.0 * (2.0 - a->poisson) * (1.0 + a->poisson) / a->young +",
     "return 1.0 / (1.0 * (2.0 - a->poisson) * (1.0 + a->poisson) / a->young +",
     ["test_tangential_stiffness_mindlin_with_rolling_coupling"]),
    ("tangential damping dropped", "o->Ft[d] = -(kt * dt_t[d]) - eta_t * vrt[d];",
     "o->Ft[d] = -(kt * dt_t[d]);", ["test_tangential_damping_decay_rate"]),
    ("moment of inertia factor", "s->I[i] = 0.4 * s->m[i] * R * R;", "s->I[i] = 0.5 * s->m[i] * R * R;",
     ["test_sliding_then_rolling_five_sevenths", "test_tangential_stiffness_mindlin_with_rolling_coupling"]),
    ("tangential torque sign (walls)", "s->M[3 * i + d] += s->R[i] * o.nxFt[d] + o.Mr[d];\n      }\n      {\n        double f[3]",
     "s->M[3 * i + d] += -s->R[i] * o.nxFt[d] + o.Mr[d];\n      }\n      {\n        double f[3]",
     ["test_sliding_then_rolling_five_sevenths"]),
    ("tangential overlap update sign", "dt_t[d] = dt_t[d] + vrt[d] * dt;", "dt_t[d] = dt_t[d] - vrt[d] * dt;",
     ["test_tangential_stiffness_mindlin_with_rolling_coupling", "test_sliding_then_rolling_five_sevenths"]),
    ("rotation term of the contact velocity", "vij[d] = (s->v[3 * i + d] - Vw[d]) + rwxn[d];",
     "vij[d] = (s->v[3 * i + d] - Vw[d]) - rwxn[d];", ["test_sliding_then_rolling_five_sevenths"]),
    ("Coulomb limit keeps the overlap", "      dt_t[d] = (o->Ft[d] + eta_t * vrt[d]) / (-kt);\n", "",
     ["test_coulomb_limit_invariant_and_continuity", "test_sliding_then_rolling_five_sevenths"]),
    ("Coulomb overlap without the damping correction",
     "dt_t[d] = (o->Ft[d] + eta_t * vrt[d]) / (-kt);", "dt_t[d] = (o->Ft[d]) / (-kt);",
     ["test_coulomb_limit_invariant_and_continuity"]),
    ("rolling torque dropped", "if (rolling == 1 && adw > 0.0)", "if (rolling == 7 && adw > 0.0)",
     ["test_rolling_resistance_deceleration"]),
    ("wall spin ignored in rolling", "dw[d] = s->w[3 * i + d] - Om[d];", "dw[d] = s->w[3 * i + d];",
     ["test_turntable_spin_up_by_rolling_torque"]),
    ("wall surface velocity reversed", "cross3(Om, arm, Vw);", "cross3(arm, Om, Vw);",
     ["test_turntable_spin_up_by_rolling_torque", "test_cylinder_static_overlap_and_drum_drag"]),
    ("translation of the wall ignored", "Vw[d] += W->velocity[d];", "Vw[d] += 0.0;",
     ["test_translating_plate_drags_sphere_to_two_sevenths"]),
    ("reaction on j missing", "s->F[3 * j + d] -= f;", "s->F[3 * j + d] -= 0.5 * f;",
     ["test_momentum_conserved_by_pair_forces"]),
    ("Euler drift instead of Verlet", "double h = 0.5 * c->dt;", "double h = 0.0 * c->dt;",
     ["test_free_fall_is_exact"]),
    ("search threshold not strict", "if (sqdist(&s->x[3 * i], &s->x[3 * j]) < rc2) {",
     "if (sqdist(&s->x[3 * i], &s->x[3 * j]) <= rc2) {", [("test_cell_search_equals_brute_force", dict(seed=1))]),
    ("search misses diagonal cells", "for (int dz = -1; dz <= 1; dz++)", "for (int dz = 0; dz <= 1; dz++)",
     [("test_cell_search_equals_brute_force", dict(seed=1))]),
    ("floating wall never switches off", "int on = s->active[i] && t >= W->t_on && t < W->t_off;",
     "int on = s->active[i] && t >= W->t_on;", ["test_floating_wall_holds_until_t_off"]),
    ("cylinder overlap sign", "double ov = R - (W->radius - rho);", "double ov = R - (rho - W->radius);",
     ["test_cylinder_static_overlap_and_drum_drag"]),
    ("annulus rim ignored", "if (rho < W->inner_radius || rho > W->radius) {", "if (rho > W->radius) {",
     ["test_annulus_face_and_rim_contact_geometry"]),
    ("tangential torque on j reversed", "s->M[3 * j + d] += s->R[j] * o.nxFt[d] - o.Mr[d];",
     "s->M[3 * j + d] += -s->R[j] * o.nxFt[d] - o.Mr[d];",
     [("test_angular_momentum_changes_only_by_the_overlap_lever", dict(poly=0.0))]),
    ("rolling torque on j not opposite", "s->M[3 * j + d] += s->R[j] * o.nxFt[d] - o.Mr[d];",
     "s->M[3 * j + d] += s->R[j] * o.nxFt[d] + o.Mr[d];",
     [("test_angular_momentum_changes_only_by_the_overlap_lever", dict(poly=0.0))]),
    ("lever of j taken from i", "s->M[3 * j + d] += s->R[j] * o.nxFt[d] - o.Mr[d];",
     "s->M[3 * j + d] += s->R[i] * o.nxFt[d] - o.Mr[d];",
     [("test_angular_momentum_changes_only_by_the_overlap_lever", dict(poly=0.3))]),
    ("wall effective mass halved", "contact_law(nrm, dn, vij, dw, vom, s->R[i], s->m[i], Yw,",
     "contact_law(nrm, dn, vij, dw, vom, s->R[i], 0.5 * s->m[i], Yw,", ["test_restitution_on_wall"]),
    ("wall damping from the particle's restitution", "double bw = damping_beta(c->wall.restitution);",
     "double bw = damping_beta(c->particle.restitution);", ["test_restitution_on_wall"]),
    ("wall friction from the particle material", "Yw, Gw, bw, c->wall.mu_slide, c->wall.mu_roll,",
     "Yw, Gw, bw, c->particle.mu_slide, c->wall.mu_roll,", ["test_sliding_then_rolling_five_sevenths"]),
    ("wall rolling friction from the particle material", "Yw, Gw, bw, c->wall.mu_slide, c->wall.mu_roll,",
     "Yw, Gw, bw, c->wall.mu_slide, c->particle.mu_roll,", ["test_rolling_resistance_deceleration"]),
    ("wall shear modulus without the wall", "double Gw = eff_shear(&c->particle, &c->wall);",
     "double Gw = eff_shear(&c->particle, &c->particle);", ["test_tangential_stiffness_mindlin_with_rolling_coupling"]),
    ("partner spin subtracted in the pair contact velocity",
     "rw[d] = s->R[i] * s->w[3 * i + d] + s->R[j] * s->w[3 * j + d];",
     "rw[d] = s->R[i] * s->w[3 * i + d] - s->R[j] * s->w[3 * j + d];",
     ["test_meshing_spins_do_not_slip_and_feel_only_rolling_resistance",
      "test_sliding_collision_tangential_impulse_is_mu_times_normal"]),
    ("rotation term of the pair contact velocity reversed", "vij[d] = (s->v[3 * i + d] - s->v[3 * j + d]) + rwxn[d];",
     "vij[d] = (s->v[3 * i + d] - s->v[3 * j + d]) - rwxn[d];",
     ["test_sliding_collision_tangential_impulse_is_mu_times_normal"]),
    ("relative spin of a pair summed", "dw[d] = s->w[3 * i + d] - s->w[3 * j + d];",
     "dw[d] = s->w[3 * i + d] + s->w[3 * j + d];",
     ["test_meshing_spins_do_not_slip_and_feel_only_rolling_resistance"]),
    ("error scales never cleared", "memset(s->Fabs, 0, sizeof(double) * n);", "memset(s->Fabs, 0, 0);",
     ["test_error_scales_of_a_sliding_sphere"]),
    ("error scale without the rolling torque", "s->Mabs[i] += s->R[i] * norm3(o.nxFt) + norm3(o.Mr);",
     "s->Mabs[i] += s->R[i] * norm3(o.nxFt);", ["test_error_scales_of_a_sliding_sphere"]),
    ("wall overlaps of different particles share a slot", "double* H = &s->Hw[(i * ORC_MAX_WALLS + k) * 3];",
     "double* H = &s->Hw[(i / ORC_MAX_WALLS + k) * 3];", ["test_spheres_that_never_meet_move_as_if_alone"]),
    ("rotation origin of a translating wall left behind", "Wt.rot_origin[d] = Wt.rot_origin[d] + Wt.velocity[d] * t;",
     "Wt.rot_origin[d] = Wt.rot_origin[d] - Wt.velocity[d] * t;", ["test_translating_turntable_carries_a_co_moving_sphere"]),
    ("floating wall still there at t_off", "t >= W->t_on && t < W->t_off;", "t >= W->t_on && t <= W->t_off;",
     ["test_floating_wall_window_is_half_open"]),
    ("floating wall late by a step", "t >= W->t_on && t < W->t_off;", "t > W->t_on && t < W->t_off;",
     ["test_floating_wall_window_is_half_open"]),
    ("cylinder axis point added", "if (W->kind == 1) { /* inside of a cylinder: distance to the mantle */\n"
     "    double rel[3] = {x[0] - W->point[0],", "if (W->kind == 1) { /* inside of a cylinder: distance to the mantle */\n"
     "    double rel[3] = {x[0] + W->point[0],", ["test_wall_contacts_are_invariant_under_translation"]),
    ("cylinder radial vector keeps the axial part",
     "double rad[3] = {rel[0] - ax * W->normal[0], rel[1] - ax * W->normal[1],",
     "double rad[3] = {rel[0] - ax * W->normal[0], rel[1] + ax * W->normal[1],",
     ["test_wall_contacts_are_invariant_under_translation"]),
    ("annulus centre added", "/* annulus: nearest point of a flat ring (face, or the rim of the hole) */\n"
     "    double rel[3] = {x[0] - W->point[0],", "/* annulus: nearest point of a flat ring (face, or the rim of the hole) */\n"
     "    double rel[3] = {x[0] + W->point[0],", ["test_wall_contacts_are_invariant_under_translation"]),
    ("Euler spin update reversed", "s->w[3 * i + d] = s->w[3 * i + d] + al * c->dt;",
     "s->w[3 * i + d] = s->w[3 * i + d] - al * c->dt;",
     ["variants.test_explicit_euler_sliding_then_rolling_five_sevenths"]),
    ("Euler never removes particles", "      s->w[3 * i + d] = s->w[3 * i + d] + al * c->dt;\n    }\n"
     "    if (s->x[3 * i + 2] < c->z_sink) s->active[i] = 0;", "      s->w[3 * i + d] = s->w[3 * i + d] + al * c->dt;\n    }\n",
     ["variants.test_explicit_euler_removes_a_sphere_below_z_sink"]),
    ("pair velocity components mixed", "vij[d] = (s->v[3 * i + d] - s->v[3 * j + d]) + rwxn[d];",
     "vij[d] = (s->v[3 * i - d] - s->v[3 * j + d]) + rwxn[d];",
     ["test_an_oblique_spinning_collision_is_rotation_invariant"]),
    ("partner spin read from the wrong particle", "rw[d] = s->R[i] * s->w[3 * i + d] + s->R[j] * s->w[3 * j + d];",
     "rw[d] = s->R[i] * s->w[3 * i + d] + s->R[j] * s->w[3 / j + d];",
     ["test_an_oblique_spinning_collision_is_rotation_invariant"]),
    ("plane contact point mirrored", "pstar[d] = x[d] - dist * W->normal[d];", "pstar[d] = x[d] + dist * W->normal[d];",
     ["test_a_paddle_turning_about_its_contact_point_does_not_drag"]),
    ("cylinder radial vector with a wrong component", "double rad[3] = {rel[0] - ax * W->normal[0],",
     "double rad[3] = {rel[0] + ax * W->normal[0],", ["test_wall_contacts_are_rotation_invariant"]),
    ("annulus in-plane offset with a wrong component",
     "double q[3] = {rel[0] - h * W->normal[0],", "double q[3] = {rel[0] + h * W->normal[0],",
     ["test_wall_contacts_are_rotation_invariant"]),
    ("rotation arm with a wrong component", "ps[1] - W->rot_origin[1]", "ps[1] + W->rot_origin[1]",
     ["test_wall_contacts_are_rotation_invariant"]),
    ("pair error scale loses the rolling torque", "s->Mabs[i] += s->R[i] * at + ar;", "s->Mabs[i] += s->R[i] * at - ar;",
     ["test_meshing_spins_do_not_slip_and_feel_only_rolling_resistance"]),
    ("overlap dropped at a search", "for (int d = 0; d < 3; d++) H[3 * k + d] = s->H[3 * a + d];",
     "for (int d = 0; d < 3; d++) H[3 * k + d] = 0.0;", ["test_trajectory_is_independent_of_the_search_cadence"]),
    ("search trigger at the full skin", "double half = 0.5 * s->cfg.skin;", "double half = 1.0 * s->cfg.skin;",
     ["test_trajectory_is_independent_of_the_search_cadence", "test_dynamic_rebuild_keeps_all_contacts_in_list"]),
    ("particles never leave",
     "    for (int d = 0; d < 3; d++) s->x[3 * i + d] = s->x[3 * i + d] + s->v[3 * i + d] * c->dt;\n"
     "    if (s->x[3 * i + 2] < c->z_sink) s->active[i] = 0;",
     "    for (int d = 0; d < 3; d++) s->x[3 * i + d] = s->x[3 * i + d] + s->v[3 * i + d] * c->dt;\n",
     ["test_particles_leave_below_z_sink_and_stay_put"]),
    ("removed particles still interact", "    if (!s->active[i] || !s->active[j]) {", "    if (0) {",
     ["test_a_removed_particle_exerts_no_force"]),
    ("constant search one step late", "return s->since_search >= s->cfg.rebuild_every;",
     "return s->since_search > s->cfg.rebuild_every;", [("test_constant_search_runs_every_n_steps", dict(every=7))]),
    # the paper's variants (pins in test_oracle_variants.py)
    ("linear stiffness exponent", "kn = 16.0 / 15.0 * sR * Ye * fifth_root(arg);",
     "kn = 16.0 / 15.0 * sR * Ye * sqrt(arg);",
     ["variants.test_linear_stiffness_gives_hertz_overlap_at_the_characteristic_speed"]),
    ("linear damping drops the 4", "eta_n = sqrt(4.0 * me * kn / lo->lin_den);",
     "eta_n = sqrt(me * kn / lo->lin_den);",
     [("variants.test_linear_damping_recovers_the_input_restitution", dict(e=0.8))]),
    ("linear model stiffer tangentially", "    kt = kn;\n    eta_t = eta_n;",
     "    kt = 2.0 * kn;\n    eta_t = eta_n;", ["test_momentum_conserved_by_pair_forces",
                                                  "variants.test_linear_tangential_stiffness_equals_normal"]),
    ("viscous rolling without |V_omega|", "o->Mr[d] = -mu_r * Re * aFn * avw * dw[d] / adw;",
     "o->Mr[d] = -mu_r * Re * aFn * dw[d] / adw;", ["variants.test_viscous_rolling_decays_exponentially"]),
    ("Euler drifts with the new velocity",
     "      s->x[3 * i + d] = s->x[3 * i + d] + s->v[3 * i + d] * c->dt;\n      s->v[3 * i + d] = s->v[3 * i + d] + a * c->dt;",
     "      s->v[3 * i + d] = s->v[3 * i + d] + a * c->dt;\n      s->x[3 * i + d] = s->x[3 * i + d] + s->v[3 * i + d] * c->dt;",
     ["variants.test_explicit_euler_free_fall_follows_the_discrete_recursion"]),
    ("translating wall moves backwards", "Wt.point[d] = Wt.point[d] + Wt.velocity[d] * t;",
     "Wt.point[d] = Wt.point[d] - Wt.velocity[d] * t;",
     ["variants.test_translating_wall_hits_and_throws_a_resting_sphere"]),
]


@pytest.mark.parametrize("name,old,new,tests", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_kill_mutant(name, old, new, tests, tmp_path):
    src = oracle.source()
    assert src.count(old) == 1, f"mutation anchor not unique: {old!r}"
    lib = oracle.compile_variant(src.replace(old, new), os.path.join(str(tmp_path), "mut.so"))
    failed = []
    with oracle.swap_library(lib):
        for t in tests:
            name_t, kw = (t, {}) if isinstance(t, str) else t
            mod = variants if name_t.startswith("variants.") else pins
            fn = getattr(mod, name_t.split(".")[-1])
            try:
                fn(**kw)
            except (AssertionError, ValueError, RuntimeError, FloatingPointError):
                failed.append(t)
    assert failed, f"mutant '{name}' survived {tests}"
