"""Planted mistakes in the oracle must be caught by its pins.

Each case copies oracle/dcem_oracle.c, plants one plausible mistake (a flipped
sign, a dropped factor, a swapped operand, a missing test), builds the copy
in a folder of its own and runs the CPU pin suites against it in a child
process (the oracle driver reads DCEM_ORACLE_SRC / DCEM_ORACLE_BUILD). The
pins are meant to fix every part of the oracle by something other than the
oracle itself (closed forms, textbook limits, invariants, brute force), so
each mutant must fail at least one of them.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dcem_oracle.c")
PINS = [os.path.join(ROOT, "tests", "test_oracle_pins.py"), os.path.join(ROOT, "tests", "test_oracle_grad_pins.py"),
        os.path.join(ROOT, "tests", "test_oracle_keller.py"), os.path.join(ROOT, "tests", "test_oracle_diffract_trans.py")]

# (name, exact text in the source, replacement). The text of each case must
# occur in the source; every occurrence is replaced.
MUTANTS = [
    # Fresnel coefficients (Snell-law forms, Brewster, normal incidence)
    ("te_sign", "*g_te = (cos_t - root) / (cos_t + root);", "*g_te = (cos_t + root) / (cos_t - root);"),
    ("tm_without_eps", "*g_tm = (ec * cos_t - root) / (ec * cos_t + root);",
     "*g_tm = (cos_t - root) / (cos_t + root);"),
    ("conductivity_sign", "double complex ec = eps_r - I * (sigma / (2.0 * M_PI * freq * EPS0));",
     "double complex ec = eps_r + I * (sigma / (2.0 * M_PI * freq * EPS0));"),
    # polarisation basis of a bounce
    ("swapped_pol_basis", "v3 pin = cross(sv, din), pout = cross(sv, dout);",
     "v3 pin = cross(sv, dout), pout = cross(sv, din);"),
    # image sources
    ("image_half_distance", "img[q] = sub(img[q - 1], scl(T->n, 2.0 * h));",
     "img[q] = sub(img[q - 1], scl(T->n, h));"),
    # reception sphere radius
    ("capture_radius", "double ae = P->rx_radius_scale * P->alpha / sqrt(3.0);",
     "double ae = P->rx_radius_scale * P->alpha / 3.0;"),
    # FP32 transform order
    ("fma_order",
     "q[r] = fmaf(m[4 * r + 0], p[0], fmaf(m[4 * r + 1], p[1], fmaf(m[4 * r + 2], p[2], m[4 * r + 3])));",
     "q[r] = fmaf(m[4 * r + 2], p[2], fmaf(m[4 * r + 1], p[1], fmaf(m[4 * r + 0], p[0], m[4 * r + 3])));"),
    # closest hit
    ("farthest_hit", "if (xs[j].t < bt) { bt = xs[j].t; best = j; }",
     "if (best < 0 || xs[j].t > bt) { bt = xs[j].t; best = j; }"),
    # occlusion of sub-segments
    ("no_occlusion", "if (occluded(S, X[j], X[j + 1], ex0, ex1, P, scale + L, &fl)) ok = 0;",
     "if (0 && occluded(S, X[j], X[j + 1], ex0, ex1, P, scale + L, &fl)) ok = 0;"),
    # amplitude (Eq. 1 with the spreading of Eq. 3)
    ("amplitude_2pi", "double complex a = (lam / (4.0 * M_PI)) * cdot(E, prx) * cexp(-I * kw * L) / L;",
     "double complex a = (lam / (2.0 * M_PI)) * cdot(E, prx) * cexp(-I * kw * L) / L;"),
    ("phase_sign", "double complex a = (lam / (4.0 * M_PI)) * cdot(E, prx) * cexp(-I * kw * L) / L;",
     "double complex a = (lam / (4.0 * M_PI)) * cdot(E, prx) * cexp(I * kw * L) / L;"),
    ("spreading_squared", "double complex a = (lam / (4.0 * M_PI)) * cdot(E, prx) * cexp(-I * kw * L) / L;",
     "double complex a = (lam / (4.0 * M_PI)) * cdot(E, prx) * cexp(-I * kw * L) / (L * L);"),
    # reflection law of the shooting step
    ("reflection_half", "d = unit(sub(d, scl(T->nh, 2.0 * dot(d, T->nh))));",
     "d = unit(sub(d, scl(T->nh, dot(d, T->nh))));"),
    # delay
    ("delay_light_speed", "out->delay_s = L / C0;", "out->delay_s = L / 3.0e8;"),
    # image of the transmitter for a reflection before a diffraction
    ("diffraction_image_half", "if (first) src = sub(T, scl(Tj->nh, 2.0 * (dot(Tj->nh, T) - cpl)));",
     "if (first) src = sub(T, scl(Tj->nh, 1.0 * (dot(Tj->nh, T) - cpl)));"),
    # the reflection after a diffraction uses the bounce basis of the outgoing leg
    ("diffraction_reflection_basis", "v3 pin = cross(sv, din), pout = cross(sv, dout);\n          int mj",
     "v3 pin = cross(sv, dout), pout = cross(sv, din);\n          int mj"),
    # diffraction of order 2 and 3: Keller points, chains in a face plane, astigmatic spreading
    ("keller_gradient_sign", "if (a >= 0) { g[a] -= ca; H[a][a] += (1.0 - ca * ca) / l; }",
     "if (a >= 0) { g[a] += ca; H[a][a] += (1.0 - ca * ca) / l; }"),
    ("keller_stalls_at_the_rounding_floor", "int at_floor = gmax < 1e-8 || fabs(gdx) <= 2e-15 * Lc;",
     "int at_floor = gmax < 1e-8;"),
    ("keller_hessian_cross_sign", "double h = -(dot(E[a]->e, E[b]->e) - ca * cb) / l;",
     "double h = (dot(E[a]->e, E[b]->e) - ca * cb) / l;"),
    ("face_plane_chains_kept", "|| in_face_plane(A, B) || in_face_plane(B, A)) ok = 0;", ") ok = 0;"),
    ("caustic_on_the_edge", "rho1 = s;\n    dir1 = ph;", "rho1 = rhoe + s;\n    dir1 = ph;"),
    ("principal_direction", "dir1 = ph;\n    rho2 = rhoe + s;", "dir1 = bd;\n    rho2 = rhoe + s;"),
    ("chain_image_half", "return sub(x, scl(Tj->nh, 2.0 * (dot(Tj->nh, x) - cpl)));",
     "return sub(x, scl(Tj->nh, 1.0 * (dot(Tj->nh, x) - cpl)));"),
    ("chain_last_reflection_dropped", "Ev = reflect_field(S, P, &S->t[ja[i]], dlast, dout, Ev);", "(void)0;"),
    # two reflections around a diffraction: the images' order, the unfolding, the field
    ("refl2_image_order", "Simg[i + 1] = mirror_in(&S->t[jb[i]], Simg[i]);",
     "Simg[i + 1] = mirror_in(&S->t[jb[nb - 1 - i]], Simg[i]);"),
    ("refl2_observer_order", "Oimg[i] = mirror_in(&S->t[ja[i]], Oimg[i + 1]);",
     "Oimg[i] = mirror_in(&S->t[ja[na - 1 - i]], Oimg[i + 1]);"),
    ("refl2_unfold_from_the_last_image", "if (!mirror_point(&S->t[jb[i]], Simg[i + 1], b, P, scale, &fl, &Yb[i])) return 0;",
     "if (!mirror_point(&S->t[jb[i]], Simg[nb], b, P, scale, &fl, &Yb[i])) return 0;"),
    ("refl2_first_reflection_dropped", "Er = reflect_field(S, P, &S->t[jb[i]], din, dout, Er);",
     "if (i == nb - 1) Er = reflect_field(S, P, &S->t[jb[i]], din, dout, Er);"),
    # a reflection between two diffractions: the receiver's image, the wavefront at the mirror
    ("mid_receiver_not_mirrored", "const v3 Rm = mirror_in(Tj, R);", "const v3 Rm = R;"),
    ("mid_reflection_dropped", "Ev = reflect_field(S, P, Tj, din, dout, Ev);", "(void)0;"),
    ("mid_principal_directions_not_mirrored", "dir1 = sub(dir1, scl(Tj->nh, 2.0 * dot(dir1, Tj->nh)));",
     "(void)0;"),
    # transmissions on the legs of a first-order diffraction
    ("diffract_trans_second_leg_loss_dropped",
     "for (int i = 0; i < n2; ++i) g *= pow(10.0, -P->trans_db[S.t[c2[i]].mat] / 20.0);", "(void)0;"),
    ("diffract_trans_crossings_reversed", "while (q > 0 && us[q - 1] > u)", "while (q > 0 && us[q - 1] < u)"),
    ("diffract_trans_opaque_crossed", "if (!P->trans_db || m < 0 || m >= S->nmat || P->trans_db[m] < 0) { bad = 1; continue; }",
     "if (!P->trans_db || m < 0 || m >= S->nmat) { bad = 1; continue; }"),
    ("multi_trans_losses_dropped",
     "for (int i = 0; i < cr->total; ++i) a *= pow(10.0, -P->trans_db[S->t[cr->id[i]].mat] / 20.0);", "(void)0;"),
    ("multi_trans_limit_ignored", "cr->id + cr->total, cr->cap - cr->total);", "cr->id + cr->total, OR_MAX_REFL - m - cr->total);"),
    ("spherical_spreading", "double complex A = csqrt(rhoe / (s * (rhoe + s))) * cexp(-I * k * s);",
     "double complex A = csqrt(ell[0] / (s * (ell[0] + s))) * cexp(-I * k * s);"),
]


def test_every_mutant_text_is_in_the_source():
    src = open(SRC).read()
    for name, old, _ in MUTANTS:
        assert old in src, f"{name}: text not found in the oracle source"


def _run_pins(tmp_path, text):
    """Builds `text` as the oracle in tmp_path and runs the pin suites on it."""
    mut = tmp_path / "dcem_oracle.c"
    mut.write_text(text)
    # the mutant must build (a build error would fail the pins for another reason)
    b = subprocess.run(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
                        "-pthread", str(mut), "-o", str(tmp_path / "check.so"), "-lm"], capture_output=True, text=True)
    assert b.returncode == 0, b.stderr
    env = dict(os.environ)
    env["DCEM_ORACLE_SRC"] = str(mut)
    env["DCEM_ORACLE_BUILD"] = str(tmp_path / "build")
    return subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-m", "not gpu", "-p", "no:cacheprovider",
                           *PINS], cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)


def test_unmodified_copy_passes_the_pins(tmp_path):
    """Control: the same route with the source unchanged passes."""
    r = _run_pins(tmp_path, open(SRC).read())
    assert r.returncode == 0, r.stdout[-2000:]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_mutant_is_caught_by_a_pin(tmp_path, name, old, new):
    src = open(SRC).read()
    assert old in src
    r = _run_pins(tmp_path, src.replace(old, new))
    assert r.returncode == 1, f"mutant {name} survived the pins (rc {r.returncode}):\n{r.stdout[-2000:]}"
