"""The oracle's pins must be able to fail.

Each case plants one plausible mistake (a flipped sign, a dropped term, a
shifted stagger, a wrong face) in a temporary copy of the oracle source, on
the CPU, and checks that the pin named beside it now fails.  Nothing here
touches a GPU.
"""
import os
import shutil
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

MUTATIONS = [
    ("boris rotation sign", "vm[1] * b[2] - vm[2] * b[1]", "vm[2] * b[1] - vm[1] * b[2]",
     "test_boris_pure_B_conserves_speed_and_rotates_2atan_b or test_boris_ExB_drift_direction"),
    ("Esirkepov dropped 1/2 term",
     "0.5 * S0[1][j] * DS[2][k] + DS[1][j] * DS[2][k] / 3.0);\n                    run += W;\n"
     "                    if (run != 0.0) fadd(s, s->J[0]",
     "0.0 * S0[1][j] * DS[2][k] + DS[1][j] * DS[2][k] / 3.0);\n                    run += W;\n"
     "                    if (run != 0.0) fadd(s, s->J[0]",
     "test_esirkepov_satisfies_continuity_exactly"),
    ("E_x stagger", "{{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}}",
     "{{0.0, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}}", "test_gather_is_exact_for_linear_fields"),
    ("Yee curl sign", "s->B[2][c] -= dt * (tBzx - tBzy);", "s->B[2][c] -= dt * (tBzx + tBzy);",
     "test_yee_plane_waves_follow_numerical_dispersion"),
    ("Hooke force sign",
     "kick[a] = 0.5 * dt * (q / m * E[a] - hooke);",
     "kick[a] = 0.5 * dt * (q / m * E[a] + hooke);",
     "test_bound_push_reproduces_taflove_recurrence"),
    ("damping sign", "rhs[r] = (1.0 - 0.5 * dt * gamma[r]) * vm[r];",
     "rhs[r] = (1.0 + 0.5 * dt * gamma[r]) * vm[r];", "test_bound_damping_factor"),
    ("damping of the wrong axis", "rhs[r] = (1.0 - 0.5 * dt * gamma[r]) * vm[r];",
     "rhs[r] = (1.0 - 0.5 * dt * gamma[(r + 1) % 3]) * vm[r];", "test_bound_anisotropic_gamma"),
    ("damping of the wrong axis in the solve",
     "L[r][c] = (r == c ? 1.0 + 0.5 * dt * gamma[r] : 0.0) - X[r][c];",
     "L[r][c] = (r == c ? 1.0 + 0.5 * dt * gamma[2 - r] : 0.0) - X[r][c];",
     "test_bound_anisotropic_gamma"),
    ("reflection not mirrored", "X1[a] = 2.0 * face - X1[a];", "X1[a] = X0[a];",
     "test_reflection_hand_computed"),
    ("source sign", "double Js = -2.0 * s->E0", "double Js = 2.0 * s->E0",
     "test_soft_source_launches_E0_pulse"),
    ("CPML coefficient sign", "*c = *b - 1.0;", "*c = 1.0 - *b;", "test_cpml_absorbs_the_pulse"),
    ("FD density of states", "return (L->dirac ? p : p * p) * f;",
     "return (L->dirac ? p : p * p * p) * f;", "test_fd_finite_temperature_sommerfeld_3d"),
    ("2D3V J_z factor", "double fz = qw * vz / (d[0] * d[1] * d[2]);",
     "double fz = 0.5 * qw * vz / (d[0] * d[1] * d[2]);",
     "test_esirkepov_satisfies_continuity_exactly"),
    ("Dirac renormalisation", "v[0] = vF * v[0] / nrm;", "v[0] = vF * v[0] / (nrm * 1.0000001);",
     "test_dirac_speed_is_vF"),
    ("Philox key increment", "k0 += 0x9E3779B9u;", "k0 += 0x9E3779B7u;",
     "test_philox_known_answers"),
    ("permittivity on the curl term only",
     "s->E[1][c] += dt / er * (c2 * (tEyz - tEyx) - s->J[1][c] / EPS0);",
     "s->E[1][c] += dt * (c2 * (tEyz - tEyx) / er - s->J[1][c] / EPS0);",
     "test_gauss_law_holds_for_D_in_a_dielectric"),
    ("permittivity not applied", "double er = s->eps_r ? s->eps_r[c] : 1.0;", "double er = 1.0;",
     "test_dielectric_half_space_fresnel"),
    ("work-function potential sign", "out[a][c] = -(phi1 - phi0) / s->d[a];",
     "out[a][c] = (phi1 - phi0) / s->d[a];",
     "test_work_function_planar_barrier_closed_form or test_potential_wall"),
    ("node vacuum fraction cell offset", "int c[3] = {i - 1 + di, j - 1 + dj,",
     "int c[3] = {i + di, j - 1 + dj,", "test_work_function_planar_barrier_closed_form"),
    ("external field on the B stagger",
     "if (s->Eext[c]) E[c] += interp(s, order, s->Eext[c], STAG_E[c], X);",
     "if (s->Eext[c]) E[c] += interp(s, order, s->Eext[c], STAG_B[c], X);",
     "test_external_field_gather_is_exact_for_linear_fields"),
    ("open edges ignored", "int edge = !outside && !s->open_edges &&", "int edge = !outside &&",
     "test_open_edges_let_particles_leave"),
    ("Lambert law without the square root", "const double ct = sqrt(u1), st = sqrt(1.0 - u1)",
     "const double ct = u1, st = sqrt(1.0 - u1 * u1)",
     "test_diffuse_reflection_follows_lambert_law_3d"),
    ("diffuse re-emission outward", "const double nin = c1[axis] > c0[axis] ? -1.0 : 1.0;",
     "const double nin = c1[axis] > c0[axis] ? 1.0 : -1.0;",
     "test_diffuse_reflection_follows_lambert_law_3d"),
    ("diffuse decision word", "diffuse = u24(r[0]) <", "diffuse = u24(r[3]) <",
     "test_diffuse_fraction_and_draw_layout"),
    ("2D law uniform in angle", "const double st = 2.0 * u1 - 1.0, ct = sqrt(1.0 - st * st);",
     "const double st = sin(PI * (u1 - 0.5)), ct = sqrt(1.0 - st * st);",
     "test_diffuse_reflection_of_dirac_carriers_is_2d_lambert"),
    ("binding tensor row", "const double o2 = a == 0 ? w2off[1] : a == 1 ? w2off[2] : w2off[2];",
     "const double o2 = a == 0 ? w2off[2] : a == 1 ? w2off[2] : w2off[2];",
     "test_bound_binding_tensor_is_rotation_covariant"),
    ("TSC central weight", "if (r < 0.5) return 0.75 - r * r;", "if (r < 0.5) return 0.7 - r * r;",
     "test_tsc_weights_hand_computed or test_tsc_esirkepov_satisfies_continuity_exactly"),
    ("TSC node window", "return order == 2 ? (int)floor(X + 0.5) - 1 : (int)floor(X);",
     "return order == 2 ? (int)floor(X) - 1 : (int)floor(X);",
     "test_tsc_weights_hand_computed or test_tsc_esirkepov_satisfies_continuity_exactly"),
    ("histogram edge", "if (E >= e_max) b = nbins;", "if (E > e_max) b = nbins;",
     "test_energy_histogram_bin_edges"),
    ("histogram energy factor", "double E = 0.5 * sp->m * ((v[0] * v[0]",
     "double E = sp->m * ((v[0] * v[0]", "test_energy_histogram_of_the_T0_fermi_sea"),
    ("Bn half-step factor", "double hdt = 0.5 * s->dt;", "double hdt = s->dt;",
     "test_gather_B_is_the_integer_step_average_of_the_eigenmode"),
    ("Bn correction sign", "s->Bn[0][c] = s->B[0][c] - hdt * (dEz_dy - dEy_dz);",
     "s->Bn[0][c] = s->B[0][c] + hdt * (dEz_dy - dEy_dz);",
     "test_gather_B_is_the_integer_step_average_of_the_eigenmode"),
    ("kinetic energy without the weight",
     "e += 0.5 * sp->m * sp->w * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);",
     "e += 0.5 * sp->m * (v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);",
     "test_diag_energies_hand_computed"),
    ("electric energy factor", "ue += 0.5 * EPS0 * s->E[a][c] * s->E[a][c] * V;",
     "ue += EPS0 * s->E[a][c] * s->E[a][c] * V;", "test_diag_energies_hand_computed"),
    ("magnetic energy with mu0 upside down", "ub += 0.5 / mu0() * s->B[a][c] * s->B[a][c] * V;",
     "ub += 0.5 * mu0() * s->B[a][c] * s->B[a][c] * V;", "test_diag_energies_hand_computed"),
    ("Dirac carriers pushed with the plasmon mass",
     "    orc_push_free(v, E, B, q, m, dt);\n    v[2] = 0.0;",
     "    orc_push_free(v, E, B, q, 2.0 * m, dt);\n    v[2] = 0.0;",
     "test_sheet_plasmon_frequency"),
]


@pytest.mark.parametrize("name,old,new,pin", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_planted_mistake_is_caught(tmp_path, name, old, new, pin):
    src = open(os.path.join(ROOT, "oracle", "pic_oracle.c")).read()
    assert old in src, f"mutation site for '{name}' not found"
    (tmp_path / "oracle").mkdir()
    (tmp_path / "oracle" / "pic_oracle.c").write_text(src.replace(old, new, 1))
    shutil.copy(os.path.join(ROOT, "oracle", "oracle.py"), tmp_path / "oracle" / "oracle.py")
    (tmp_path / "oracle" / "__init__.py").write_text("")
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), tmp_path / "tests" / "golden")
    for f in ("test_oracle_pins.py", "conftest.py"):
        shutil.copy(os.path.join(ROOT, "tests", f), tmp_path / "tests" / f)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                        "tests/test_oracle_pins.py", "-k", pin], cwd=tmp_path,
                       capture_output=True, text=True, timeout=600)
    assert r.returncode == 1 and "failed" in r.stdout, (name, r.stdout[-2000:])
