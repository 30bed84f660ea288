"""The oracle's pins catch plausible mistakes: each case plants one mistake
(a wrong coefficient, a flipped sign or comparison, a dropped term, a
transposed operand) in a copy of the oracle source, builds it, and runs the
pin suites against the copy, which must fail.  CPU only; the planted copies
live in a temporary directory."""
import os
import subprocess
import sys

import pytest

import oracle as O

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PINS = ["tests/test_oracle_primitives.py", "tests/test_oracle_traversal.py",
        "tests/test_oracle_grad.py", "tests/test_oracle_normals.py", "tests/test_oracle_quadratic.py",
        "tests/test_oracle_counts.py", "tests/test_oracle_thick.py"]

MUTATIONS = {
    "split_dp_coefficient": ("*dp = add4(add4(mul4(0.375, c->t0)", "*dp = add4(add4(mul4(0.125, c->t0)"),
    "split_tc_sign": ("*tc = add4(add4(mul4(-0.125, c->t0)", "*tc = add4(add4(mul4(0.125, c->t0)"),
    "right_child_t1": ("c->t1 = mul4(0.5, c->t1);", "c->t1 = mul4(0.5, c->t0);"),
    "left_child_t0": ("c->t0 = mul4(0.5, c->t0);", "c->t0 = mul4(0.25, c->t0);"),
    "go_right_flipped": ("go_right = (tp > c0) != (tc.z > 0.0);", "go_right = (tp > c0) == (tc.z > 0.0);"),
    "interval_update_side": ("if (tp > c0) tmax = dmin(tmax, tp);", "if (tp < c0) tmax = dmin(tmax, tp);"),
    "both_hit_dropped": ("if (both) bits ^= size;", "(void)both;"),
    "leaf_t_unclamped": ("t = dmax(c0, tmin);\n                hit = 1;", "t = c0;\n                hit = 1;"),
    "cylinder_tcpa_sign": ("double tcpa = p.z - a.z *", "double tcpa = p.z + a.z *"),
    "cylinder_s_term": ("sqrt(e * (a.z * a.z + g) / g)", "sqrt(e * (a.z * a.z) / g)"),
    "radius_drops_distance": ("return sqrt(m) + rmax;", "return rmax;"),
    "radius_drops_t1w": ("dmax(c->d.w, c->d.w - c->t1.w)", "dmax(c->d.w, c->d.w)"),
    "slab_start_sign": ("if (c->t0.z > 0.0) lo = dmax(lo, t);", "if (c->t0.z < 0.0) lo = dmax(lo, t);"),
    "jump_up_mask": ("start &= ~(size - 1u);", "start &= ~(size);"),
    "recompute_t1_at_u0": ("c->t1 = mul4(u1 - u0, bez_deriv3(Q, u1));", "c->t1 = mul4(u1 - u0, bez_deriv3(Q, u0));"),
    "u_interval": ("h->u = u0 + ul * (u1 - u0);", "h->u = u0 + ul * (u1 + u0);"),
    "frame_transposed": ("Q[k].y = q[0] * r->e2[0] + q[1] * r->e2[1] + q[2] * r->e2[2];",
                         "Q[k].y = q[0] * r->e2[0] + q[1] * r->e1[1] + q[2] * r->e2[2];"),
    "constraint_operand": ("dot3(p31, p10) >= 0.0 && dot3(p31, p32) >= 0.0",
                           "dot3(p32, p10) >= 0.0 && dot3(p31, p32) >= 0.0"),
    "grad_radius_sign": ("grad[4 * k + 3] = -(a2 * (-2.0 * c.w * B[k]));",
                         "grad[4 * k + 3] = (a2 * (-2.0 * c.w * B[k]));"),
    "grad_dB": ("v4 g1 = sub4(mul4(dB[k], e), mul4(B[k], d1));", "v4 g1 = sub4(mul4(B[k], e), mul4(B[k], d1));"),
    "limit_G2_radius": ("*h = dot3(e, e) - c.w * c.w;", "*h = dot3(e, e) - c.w;"),
    "normal_axis_point_sign": ("double xx = -ap.x, yy = -ap.y, zz = t - ap.z;",
                               "double xx = ap.x, yy = -ap.y, zz = t - ap.z;"),
    "normal_frame_swapped": ("n[i] = xx * r.e1[i] + yy * r.e2[i] + zz * r.w[i];",
                             "n[i] = xx * r.e2[i] + yy * r.e1[i] + zz * r.w[i];"),
    "normal_axis_point_unprojected": ("v4 ap = add4(c.p, mul4(ul, c.d));", "v4 ap = c.p;"),
    "normal_cap_points": ("int a = cap0 ? 0 : 3, b = cap0 ? 1 : 2;", "int a = cap0 ? 0 : 3, b = cap0 ? 1 : 1;"),
    "box_dilation_dropped": ("lo[a] = dmin(lo[a], v[a] - q[k].w);", "lo[a] = dmin(lo[a], v[a]);"),
    "box_retest_uncounted": ("        *count += 1;\n        if (box_hit(b, *best))", "        if (box_hit(b, *best))"),
    "thick_drops_radius": ("poly_t Pq = padd(pmul(pmul(D, D), T), X, -rbar * rbar);",
                           "poly_t Pq = padd(pmul(pmul(D, D), T), X, -rbar);"),
    "thick_end_normal": ("v4 nrm[2] = {sub4(P[1], P[0]), sub4(P[3], P[2])};",
                         "v4 nrm[2] = {sub4(P[1], P[0]), sub4(P[3], P[1])};"),
    "quadratic_elevation_weight": ("cp16[4 + a] = (p0 + 2.0 * p1) / 3.0;", "cp16[4 + a] = (2.0 * p0 + p1) / 3.0;"),
    "quadratic_constraint_sign": ("return dot3(a, b) <= 0.0;", "return dot3(a, b) >= 0.0;"),
    "normal_cap_plane_sign": ("cap0 = dot3(sub4(x, Q[0]), a0) / sqrt(dot3(a0, a0)) >= -tol;",
                              "cap0 = dot3(sub4(x, Q[0]), a0) / sqrt(dot3(a0, a0)) <= -tol;"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(O._SRC).read()
    assert src.count(old) == 1, "mutation anchor not found: %s" % name
    mut = tmp_path / "fiber_oracle_mut.c"
    mut.write_text(src.replace(old, new))
    so = O.build(src=str(mut), out=str(tmp_path / "libmut.so"))
    env = dict(os.environ, FIBER_ORACLE_LIB=so)
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + PINS,
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, "planted mistake %s passed every pin" % name
