"""The pins catch plausible mistakes: each case plants one mistake in a copy of
the oracle's source (on the CPU), builds it, and runs the pin suite against it;
at least one pin must fail.  The unmodified source must pass."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "dare_oracle.c")

MUTANTS = {
    "in-plane term without absolute value (Eq. 1)":
        ("double d_inplane = fabs(x_s[0] * c->x_r[0] + x_s[1] * c->x_r[1] + x_s[2] * c->x_r[2]);",
         "double d_inplane = (x_s[0] * c->x_r[0] + x_s[1] * c->x_r[1] + x_s[2] * c->x_r[2]);"),
    "normal term with absolute value (Eq. 1)":
        ("double d_normal = n_s[0] * c->n_r[0] + n_s[1] * c->n_r[1] + n_s[2] * c->n_r[2];",
         "double d_normal = fabs(n_s[0] * c->n_r[0] + n_s[1] * c->n_r[1] + n_s[2] * c->n_r[2]);"),
    "Eq. 2 constants swapped":
        ("return exp(p->k_normal * (d_normal - 1.0) + p->k_inplane * (d_inplane - 1.0));",
         "return exp(p->k_inplane * (d_normal - 1.0) + p->k_normal * (d_inplane - 1.0));"),
    "Eq. 2 in-plane term dropped":
        ("return exp(p->k_normal * (d_normal - 1.0) + p->k_inplane * (d_inplane - 1.0));",
         "return exp(p->k_normal * (d_normal - 1.0));"),
    "threshold on the wrong term":
        ("if (c->use_thr_i && d_inplane < c->cos_i) return 0.0;",
         "if (c->use_thr_i && d_normal < c->cos_i) return 0.0;"),
    "trilinear weight reuses the x distance":
        ("t = (1.0 - fabs(dx) / R) * (1.0 - fabs(dy) / R) * (1.0 - fabs(dz) / R);",
         "t = (1.0 - fabs(dx) / R) * (1.0 - fabs(dx) / R) * (1.0 - fabs(dz) / R);"),
    "TENT window one voxel too wide":
        ("lo[a] = f - R + 1; hi[a] = f + R;\n        }\n    }\n    double num",
         "lo[a] = f - R; hi[a] = f + R;\n        }\n    }\n    double num"),
    "voxelisation floors instead of rounding":
        ("c[a] = fix_floor(G + FIX_ONE / 2); /* nearest voxel, ties up */",
         "c[a] = fix_floor(G); /* nearest voxel, ties up */"),
    "beam read from the lateral column":
        ("quat_axis(q, p->normal_axis == 1 ? 2 : 1, n_s);", "quat_axis(q, p->normal_axis == 1 ? 2 : 0, n_s);"),
    "volume rotation not transposed":
        ("R[3 * r + c] = V[0 * 4 + r] * T[0 * 4 + c] + V[1 * 4 + r] * T[1 * 4 + c] + V[2 * 4 + r] * T[2 * 4 + c];",
         "R[3 * r + c] = V[r * 4 + 0] * T[0 * 4 + c] + V[r * 4 + 1] * T[1 * 4 + c] + V[r * 4 + 2] * T[2 * 4 + c];"),
    "pixel centring term dropped":
        ("out[r] = fix_round((tm[r] - half_w * c0[r]) / h);", "out[r] = fix_round(tm[r] / h);"),
    "capacity tie-break reversed":
        ("return x->frame < y->frame ? -1 : (x->frame > y->frame);",
         "return x->frame > y->frame ? -1 : (x->frame < y->frame);"),
    "bf16 storage truncates":
        ("b = (b + 0x7FFFu + lsb) & 0xFFFF0000u;", "b = b & 0xFFFF0000u;"),
    "fan steering angle sign flipped":
        ("double alpha = (dx == 0.0 && dy == 0.0) ? 0.0 : atan2(-dx, dy);",
         "double alpha = (dx == 0.0 && dy == 0.0) ? 0.0 : atan2(dx, dy);"),
    "fan turn applied before the frame rotation":
        ("    quat_mul(q, turn, out);\n}", "    quat_mul(turn, q, out);\n}"),
    "fan turn quaternion without the half angle":
        ("double turn[4] = {cos(0.5 * alpha), 0.0, 0.0, sin(0.5 * alpha)};",
         "double turn[4] = {cos(alpha), 0.0, 0.0, sin(alpha)};"),
    "sample fan taken at the voxel index, not its centre":
        ("w[r] = V[4 * r + 0] * (h * c[0]) + V[4 * r + 1] * (h * c[1]) + V[4 * r + 2] * (h * c[2]) +",
         "w[r] = V[4 * r + 0] * c[0] + V[4 * r + 1] * c[1] + V[4 * r + 2] * c[2] +"),
    "fan apex coordinates swapped":
        ("steer(fq + 4 * (size_t)fr, p[0], p[1], apex[2 * fr], apex[2 * fr + 1], v->quat + 4 * out);",
         "steer(fq + 4 * (size_t)fr, p[0], p[1], apex[2 * fr + 1], apex[2 * fr], v->quat + 4 * out);"),
    "voxel centre rotated into the frame without transposing":
        ("p[k] = T[0 * 4 + k] * (w[0] - T[3]) + T[1 * 4 + k] * (w[1] - T[7]) +\n"
         "                                   T[2 * 4 + k] * (w[2] - T[11]);",
         "p[k] = T[k * 4 + 0] * (w[0] - T[3]) + T[k * 4 + 1] * (w[1] - T[7]) +\n"
         "                                   T[k * 4 + 2] * (w[2] - T[11]);"),
    "virtual fan measured from the image corner":
        ("steer(c0->q, ((double)x - c0->half_w) * c0->sx,", "steer(c0->q, (double)x * c0->sx,"),
    "virtual fan leaves the lateral axis unturned":
        ("quat_axis(qp, 0, cp.x_r);", "quat_axis(c0->q, 0, cp.x_r);"),
    "pixel mask ignored":
        ("if (pixel_mask && !pixel_mask[(size_t)y * W + x]) continue;", ""),
    "hole weights without the square root":
        ("const double w = 1.0 / sqrt((double)(dx * dx + dy * dy + dz * dz));",
         "const double w = 1.0 / (double)(dx * dx + dy * dy + dz * dz);"),
    "hole filling ignores min_neighbours":
        ("filled[i] = (n >= min_neighbours && n > 0) ? num / den : NAN;", "filled[i] = n > 0 ? num / den : NAN;"),
    "hole filling cube one voxel short":
        ("        for (int64_t dz = -r; dz <= r; ++dz)\n            for (int64_t dy = -r; dy <= r; ++dy)\n"
         "                for (int64_t dx = -r; dx <= r; ++dx) {",
         "        for (int64_t dz = -r; dz < r; ++dz)\n            for (int64_t dy = -r; dy <= r; ++dy)\n"
         "                for (int64_t dx = -r; dx <= r; ++dx) {"),
    "scalar-volume reslice blends empty corners as zero":
        ("const double S = values[cx + (int64_t)dims[0] * (cy + (int64_t)dims[1] * cz)];\n                if (isnan(S)) continue;",
         "const double S0 = values[cx + (int64_t)dims[0] * (cy + (int64_t)dims[1] * cz)];\n"
         "                const double S = isnan(S0) ? 0.0 : S0;"),
    "per-pixel weight missing from the denominator":
        ("                    den += t * w * m;", "                    den += t * w;"),
    "unassigned when the numerator is zero":
        ("    if (den > 0) {\n        *out = num / den;", "    if (num > 0) {\n        *out = num / den;"),
}


def _run_pins(lib_path):
    env = dict(os.environ, DARE_ORACLE_LIB=lib_path)
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=600)
    return r.returncode, r.stdout[-2000:]


def _build(src_text, tmp_path, name):
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src_text)
    subprocess.run(["gcc", "-O1", "-fPIC", "-shared", "-fopenmp", "-std=gnu11", "-ffp-contract=off", "-o", str(so),
                    str(c), "-lm"], check=True)
    return str(so)


@pytest.mark.slow
def test_unmodified_oracle_passes(tmp_path):
    rc, out = _run_pins(_build(open(SRC).read(), tmp_path, "clean"))
    assert rc == 0, out


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation site not unique: {name}"
    rc, out = _run_pins(_build(src.replace(old, new), tmp_path, "mutant"))
    assert rc != 0, f"no pin caught: {name}\n{out}"
