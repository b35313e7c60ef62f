"""Planted-slip check of the oracle's pins (test infrastructure).

Each entry below is a plausible mistake in ``oracle.cpp``: a swapped index,
a wrong sign, a dropped term, an off-by-one, a transposed operand, a wrong
constant.  For each one this script writes a copy of ``oracle.cpp`` with that
one change into a temporary directory, compiles it with the oracle's flags,
and runs the CPU pin tests against the copy (``RG_ORACLE_LIB`` points the
oracle's loader at it).  A slip that no pin test fails is reported; the
script exits 1 if there is one.  The oracle's own source is never modified.

Three plausible changes are left out because they do not change any
result: dropping the zero-area early return (the watertight determinant of
such a triangle is already exactly 0), reporting a miss's u, v without the
hit check (a miss's u, v are already 0), and starting the shadow segment at
the offset distance instead of 0 (an occluder that close to the offset
origin cannot be placed below the surface the camera sees).

Usage: ``python oracle/plant_slips.py [-j JOBS] [NAME_SUBSTRING ...]``
(about 10 s of CPU per slip).
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import os
import subprocess
import sys
import tempfile

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "oracle.cpp")
PIN_TESTS = ["tests/test_oracle_pins.py", "tests/test_oracle_ambiguity.py", "tests/test_oracle_sah.py",
             "tests/test_oracle_fxaa.py"]

# (name, text in oracle.cpp, text it becomes)
SLIPS = [
    ('bary swap',
     'on_tri(Cand{t, k, prim, strict, inner, b1, b2,',
     'on_tri(Cand{t, k, prim, strict, inner, b2, b1,'),
    ('tie inst reversed',
     '(ct == bt && (c.inst < best.inst ||',
     '(ct == bt && (c.inst > best.inst ||'),
    ('tie prim reversed',
     '(c.inst == best.inst && c.prim < best.prim)));',
     '(c.inst == best.inst && c.prim > best.prim)));'),
    ('farthest hit',
     'bool better = !have || ct < bt ||',
     'bool better = !have || ct > bt ||'),
    ('open tmin',
     'bool strict = inside && t >= t0 && t <= t1_cull;',
     'bool strict = inside && t > t0 && t <= t1_cull;'),
    ('open tmax',
     'if (c.strict && c.t <= tmax) {',
     'if (c.strict && c.t < tmax) {'),
    ('renormalised dir',
     'V3 oo = xform_point(I.Minv, o), dd = xform_dir(I.Minv, d);',
     'V3 oo = xform_point(I.Minv, o), dd = normalize(xform_dir(I.Minv, d));'),
    ('M for Minv',
     'V3 oo = xform_point(I.Minv, o), dd = xform_dir(I.Minv, d);',
     'V3 oo = xform_point(I.M, o), dd = xform_dir(I.M, d);'),
    ('normal not transposed',
     'V3 nw{I.Minv[0] * n.x + I.Minv[4] * n.y + I.Minv[8] * n.z, I.Minv[1] * n.x + I.Minv[5] * n.y + I.Minv[9] * n.z,',
     'V3 nw{I.Minv[0] * n.x + I.Minv[1] * n.y + I.Minv[2] * n.z, I.Minv[4] * n.x + I.Minv[5] * n.y + I.Minv[6] * n.z,'),
    ('no ambient',
     'V3 L = S.ambient * a;',
     'V3 L{0, 0, 0};'),
    ('no Lambert clamp',
     'if (c <= 0) continue;',
     'if (c < -2) continue;'),
    ('shadow past light',
     'bool occ = Q.any(os, ld, 0.0, dist - eps, false, &sa);',
     'bool occ = Q.any(os, ld, 0.0, INFINITY, false, &sa);'),
    ('reflect sign',
     'V3 reflect_dir(V3 d, V3 nf) { return normalize(d - (2.0 * dot(d, nf)) * nf); }',
     'V3 reflect_dir(V3 d, V3 nf) { return normalize(d + (2.0 * dot(d, nf)) * nf); }'),
    ('snell inverted',
     'double eta = entering ? 1.0 / ior : ior;',
     'double eta = entering ? ior : 1.0 / ior;'),
    ('TIR never',
     'if (k < 0) return false;',
     'if (k < 0) k = 0;'),
    ('schlick exponent',
     'std::pow(1 - c, 5)',
     'std::pow(1 - c, 4)'),
    ('schlick cosine side',
     'double c = entering ? ci : sk;',
     'double c = ci;'),
    ('R0 wrong',
     'double R0 = ((1 - ior) / (1 + ior)) * ((1 - ior) / (1 + ior));',
     'double R0 = ((1 - ior) / (1 + ior));'),
    ('depth off by one',
     'if (depth >= max_depth) return {0, 0, 0};',
     'if (depth > max_depth) return {0, 0, 0};'),
    ('refraction offset side',
     'V3 Lt = trace(p - eps * nf, T, depth + 1, nullptr);',
     'V3 Lt = trace(p + eps * nf, T, depth + 1, nullptr);'),
    ('fresnel weights swapped',
     'return R * Lr + (1 - R) * Lt;',
     'return (1 - R) * Lr + R * Lt;'),
    ('camera rows flipped',
     'double py = (1.0 - 2.0 * (y + 0.5) / h) * th;',
     'double py = (2.0 * (y + 0.5) / h - 1.0) * th;'),
    ('camera no aspect',
     'double px = (2.0 * (x + 0.5) / w - 1.0) * aspect * th;',
     'double px = (2.0 * (x + 0.5) / w - 1.0) * th;'),
    ('camera right flipped',
     'V3 R = normalize(cross(F, up));',
     'V3 R = normalize(cross(up, F));'),
    ('camera full fov',
     'double th = std::tan(0.5 * (double)cam[9] * M_PI / 180.0);',
     'double th = std::tan((double)cam[9] * M_PI / 180.0);'),
    ('camera pixel corner',
     'double px = (2.0 * (x + 0.5) / w - 1.0) * aspect * th;',
     'double px = (2.0 * (x + 0.0) / w - 1.0) * aspect * th;'),
    ('morton x/z swapped',
     'code |= ((x >> i) & 1ull) << (3 * i + 2);',
     'code |= ((x >> i) & 1ull) << (3 * i);'),
    ('karras >=',
     'while (g + 1 <= l - 1 && delta(k, n, f, g + 1) > dn) ++g;',
     'while (g + 1 <= l - 1 && delta(k, n, f, g + 1) >= dn) ++g;'),
    ('unstable sort',
     'std::stable_sort(perm, perm + n,',
     'std::sort(perm, perm + n,'),
    ('arvo lo rounding up',
     'std::fesetround(FE_DOWNWARD);\n            volatile float s = 0.0f;',
     'std::fesetround(FE_UPWARD);\n            volatile float s = 0.0f;'),
    ('arvo min->max',
     'float mn = std::min((float)p0, (float)p1);',
     'float mn = std::max((float)p0, (float)p1);'),
    ('sphere radius unscaled',
     'volatile float R = r * norm;',
     'volatile float R = r;'),
    ('grazing inverted',
     'bool grazing = cosv * kGrazeInv < 1.0;',
     'bool grazing = cosv * kGrazeInv > 1.0;'),
    ('anyhit open tmax',
     'if (c.strict && c.t >= tmin && c.t <= tmax) strict_blocked = true;',
     'if (c.strict && c.t >= tmin && c.t < tmax) strict_blocked = true;'),
    ('back faces missed',
     'bool inside = (w.U >= 0 && w.V >= 0 && w.W >= 0) || (w.U <= 0 && w.V <= 0 && w.W <= 0);',
     'bool inside = (w.U >= 0 && w.V >= 0 && w.W >= 0);'),
    ('watertight W sign',
     'w.W = Bx * Ay - By * Ax;',
     'w.W = By * Ax - Bx * Ay;'),
    ('tri bounds lo=hi',
     'lo = std::min(lo, x);',
     'lo = std::max(lo, x);'),
    ('morton per-axis scale',
     'if (cmax[a] > cmin[a] && e > ext) ext = e;',
     'if (cmax[a] > cmin[a] && e < ext) ext = e;'),
    ('fxaa luma weights',
     '0.299f * ch(x, y, 0) + 0.587f * ch(x, y, 1) + 0.114f * ch(x, y, 2)',
     '0.587f * ch(x, y, 0) + 0.299f * ch(x, y, 1) + 0.114f * ch(x, y, 2)'),
    ('fxaa no sqrt',
     'return std::sqrt(v > 0.0f ? v : 0.0f);',
     'return v > 0.0f ? v : 0.0f;'),
    ('fxaa threshold rel',
     'const float kEdgeMin = 0.0312f, kEdgeRel = 0.125f, kSubpix = 0.75f;',
     'const float kEdgeMin = 0.0312f, kEdgeRel = 0.25f, kSubpix = 0.75f;'),
    ('fxaa subpix',
     'const float kEdgeMin = 0.0312f, kEdgeRel = 0.125f, kSubpix = 0.75f;',
     'const float kEdgeMin = 0.0312f, kEdgeRel = 0.125f, kSubpix = 0.5f;'),
    ('fxaa orientation',
     'const bool horiz = eH >= eV;',
     'const bool horiz = eH > eV;'),
    ('fxaa orientation swap',
     'const bool horiz = eH >= eV;',
     'const bool horiz = eH < eV;'),
    ('fxaa side',
     'const bool neg = std::fabs(g1) >= std::fabs(g2);',
     'const bool neg = std::fabs(g1) < std::fabs(g2);'),
    ('fxaa gradient scale',
     'const float gs = 0.25f * std::max(std::fabs(g1), std::fabs(g2));',
     'const float gs = 0.5f * std::max(std::fabs(g1), std::fabs(g2));'),
    ('fxaa step sched',
     '{1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.5f, 2.0f, 2.0f, 2.0f, 2.0f, 4.0f, 8.0f}',
     '{1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 2.0f, 2.0f, 2.0f, 2.0f, 4.0f, 8.0f}'),
    ('fxaa offset sign',
     '? 0.5f - dmin / len : 0.0f;',
     '? 0.5f - dmin / len : 0.5f;'),
    ('fxaa span cond',
     'const float off = ((lM < lLocal) != (eNear < 0.0f))',
     'const float off = ((lM < lLocal) == (eNear < 0.0f))'),
    ('fxaa avg weights',
     'const float avg = (2.0f * sum4 + sumC) / 12.0f;',
     'const float avg = (sum4 + sumC) / 8.0f;'),
    ('fxaa smoothstep',
     'sp = ((3.0f - 2.0f * sp) * sp) * sp;',
     'sp = sp;'),
    ('fxaa max->min',
     'const float f = std::max(off, sub);',
     'const float f = std::min(off, sub);'),
    ('fxaa clamp edge',
     'int cx(int x) const { return x < 0 ? 0 : (x >= w ? w - 1 : x); }',
     'int cx(int x) const { return x < 0 ? 0 : (x >= w ? 0 : x); }'),
    ('fxaa keeps alpha',
     'for (int c = 0; c < 3; ++c) out[c] = I.sample(ox, oy, c);',
     'for (int c = 0; c < 4; ++c) out[c] = I.sample(ox, oy, c);'),
    ('fxaa half pixel',
     'const float sx = horiz ? fx : fx + 0.5f * sgn, sy = horiz ? fy + 0.5f * sgn : fy;',
     'const float sx = horiz ? fx : fx + 1.0f * sgn, sy = horiz ? fy + 1.0f * sgn : fy;'),
    ('anyhit record',
     'if (inst) inst[i] = occ ? 0u : 0xFFFFFFFFu;',
     'if (inst) inst[i] = occ ? 0xFFFFFFFFu : 0u;'),
    ('amb kappa ignored',
     'double eta = kappa * EPS32 * (E0 + std::fabs(t) * E1 + m.vmax);',
     'double eta = EPS32 * (E0 + std::fabs(t) * E1 + m.vmax);'),
    ('amb no vmax',
     'double eta = kappa * EPS32 * (E0 + std::fabs(t) * E1 + m.vmax);',
     'double eta = kappa * EPS32 * (E0 + std::fabs(t) * E1);'),
    ('amb near-tie check off',
     'if (c.t <= best.t + best.tau + c.tau) { amb = true; break; }',
     'if (c.t < best.t) { amb = true; break; }'),
    ('amb inner ignored',
     'bool amb = !best.inner || best.t - best.tau < tmin || best.t + best.tau > tmax;',
     'bool amb = best.t - best.tau < tmin || best.t + best.tau > tmax;'),
    ('anyhit amb',
     '*ambiguous = outer_blocked != inner_blocked;',
     '*ambiguous = false;'),
    ('sah cost count',
     'const float cost = half_area(llo, lhi) * (float)cl + half_area(rlo, rhi) * (float)cr;',
     'const float cost = half_area(llo, lhi) + half_area(rlo, rhi);'),
    ('sah bins 15',
     'return v < 16.0f ? (int)v : 15;',
     'return v < 15.0f ? (int)v : 14;'),
    ('sah tie last',
     'if (cost < best) {',
     'if (cost <= best) {'),
    ('sah halving off',
     'const bool left = best_axis < 0 ? (p - R.b < nl) : (bin(prim[p], best_axis) < best_split);',
     'const bool left = best_axis < 0 ? (p - R.b <= nl) : (bin(prim[p], best_axis) < best_split);'),
    ('sah half area',
     'return (dx * dy + dy * dz) + dz * dx;',
     'return (dx * dy + dy * dz);'),
    ('range boxes',
     'float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};',
     'float b[6] = {0, 0, 0, -INFINITY, -INFINITY, -INFINITY};'),
    ('bound r2 centre',
     'for (int j = 0; j < 3; ++j) c[j] = (a[j] + a[3 + j]) * 0.5f;',
     'for (int j = 0; j < 3; ++j) c[j] = a[j];'),
    ('eps scale',
     'double eps = 1e-4 * std::max(1.0, amax(p));',
     'double eps = 1e-3 * std::max(1.0, amax(p));'),
    ('shadow origin below',
     'V3 os = p + eps * nf;',
     'V3 os = p - eps * nf;'),
    ('mirror origin no offset',
     'V3 Lr = trace(p + eps * nf, r, depth + 1, nullptr);\n            return {a.x * Lr.x, a.y * Lr.y, a.z * Lr.z};',
     'V3 Lr = trace(p, r, depth + 1, nullptr);\n            return {a.x * Lr.x, a.y * Lr.y, a.z * Lr.z};'),
    ('ambient not albedo',
     'V3 L = S.ambient * a;',
     'V3 L{S.ambient, S.ambient, S.ambient};'),
    ('light channel mix',
     'L = L + V3{a.x * I_l.x * c, a.y * I_l.y * c, a.z * I_l.z * c};',
     'L = L + V3{a.x * I_l.x * c, a.y * I_l.x * c, a.z * I_l.x * c};'),
    ('albedo channel mix',
     'L = L + V3{a.x * I_l.x * c, a.y * I_l.y * c, a.z * I_l.z * c};',
     'L = L + V3{a.x * I_l.x * c, a.x * I_l.y * c, a.x * I_l.z * c};'),
    ('mirror tint channel',
     'return {a.x * Lr.x, a.y * Lr.y, a.z * Lr.z};',
     'return {a.x * Lr.x, a.x * Lr.y, a.x * Lr.z};'),
    ('mirror untinted',
     'return {a.x * Lr.x, a.y * Lr.y, a.z * Lr.z};',
     'return Lr;'),
    ('camera up flipped',
     'V3 U = cross(R, F);',
     'V3 U = cross(F, R);'),
    ('TIR reflect offset',
     'return trace(p + eps * nf, r, depth + 1, nullptr);  // total internal reflection',
     'return trace(p - eps * nf, r, depth + 1, nullptr);  // total internal reflection'),
    ('glass depth',
     'if (depth >= max_depth) return {0, 0, 0};',
     'if (depth >= max_depth && type == 1) return {0, 0, 0};'),
    ('secondary hit flag',
     'if (hit_out) *hit_out = h.hit;',
     'if (hit_out) *hit_out = true;'),
]


def run_one(slip, text):
    from oracle import CXXFLAGS   # the oracle's own compiler flags
    name, old, new = slip
    if old not in text:
        return name, "not found"
    with tempfile.TemporaryDirectory() as tmp:
        src = os.path.join(tmp, "oracle.cpp")
        lib = os.path.join(tmp, "liboracle.so")
        with open(src, "w") as f:
            f.write(text.replace(old, new, 1))
        b = subprocess.run(["g++", *CXXFLAGS, "-o", lib, src, "-lpthread"], capture_output=True, text=True)
        if b.returncode:
            return name, "does not compile"
        env = dict(os.environ, RG_ORACLE_LIB=lib)
        t = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider", *PIN_TESTS],
                           cwd=ROOT, env=env, capture_output=True, text=True)
        return name, "caught" if t.returncode else "SURVIVED"


def main():
    p = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    p.add_argument("-j", "--jobs", type=int, default=max(1, (os.cpu_count() or 2) // 2))
    p.add_argument("names", nargs="*")
    args = p.parse_args()
    sys.path.insert(0, ROOT)
    text = open(SRC).read()
    slips = [s for s in SLIPS if not args.names or any(n in s[0] for n in args.names)]
    with cf.ThreadPoolExecutor(args.jobs) as ex:
        results = list(ex.map(lambda s: run_one(s, text), slips))
    width = max(len(n) for n, _ in results)
    for name, verdict in results:
        print(f"{name:<{width}}  {verdict}")
    bad = [n for n, v in results if v != "caught"]
    print(f"{len(results) - len(bad)} of {len(results)} slips caught")
    return 1 if bad else 0


if __name__ == "__main__":
    sys.exit(main())
