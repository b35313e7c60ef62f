// Oracle: a plain, slow CPU reference of the ray tracer's hot path.
//
// TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
// call this file; only the tests, the smoke check and the benchmark's CPU
// baseline do.  It shares no code, header or constant table with the CUDA
// library: its only common ground with it is the float32/uint32 input arrays
// produced by the seeded scene generators.
//
// What it computes, and where each piece comes from:
//
//  * The two-level acceleration structure (paper Sec. 1: a two-layered
//    structure built from the models' vertices and their transformation
//    matrices).  The build steps of the CUDA path (Morton codes, stable sort,
//    Karras hierarchy, box refit, instance boxes) are restated here in their
//    plain definitions, in float32 where the product computes in float32, so
//    that their results can be compared bit for bit:
//      - Morton codes: centroids quantised on one cubic grid (a single scale
//        from the largest centroid extent), bits interleaved x,y,z (MSB first).
//      - Sort: std::stable_sort (not a radix sort).
//      - Hierarchy: top-down recursive split at the highest differing bit of
//        (key, index) (Karras 2012, Sec. 4 defines the same tree bottom-up).
//      - Node boxes: the union of the leaf boxes in each node's key range
//        (not a bottom-up climb).
//      - Instance boxes: Arvo (Graphics Gems 1990) transform of the object
//        box with directed rounding, emulated with fesetround.
//      - The trace-speed BLAS hierarchy (binned surface-area heuristic,
//        MacDonald & Booth 1990 for the cost, Wald 2007 for binning): a plain
//        top-down recursion over the Morton order (orc_sah_build).  The paper
//        leaves acceleration structures to the driver, so this hierarchy is a
//        choice of the implementation; the oracle states it so that the
//        product's build can be compared with it bit for bit.
//  * Ray queries (paper Sec. 1: closest-hit, any-hit and miss per ray), in
//    float64 on an independent object-median BVH (or brute force), using the
//    watertight ray/triangle test of Woop, Benthin & Wald (JCGT 2013).  The
//    nearest hit is chosen on the exact distances rounded to float32, the
//    precision of the hit records (equal float32 t: smaller instance, then
//    smaller primitive), so exact ties such as coplanar surfaces have one
//    answer that does not depend on how float64 rounds them.  Each
//    ray also gets an "ambiguous" flag: the float32 path may legitimately
//    differ from the exact answer when another triangle lies within the
//    float32 error bound (see orc_trace).
//  * Whitted shading with shadows, reflection and refraction (paper Sec. 2.1),
//    recursive, per pixel, in float64.
//  * FXAA on the rendered image (paper Sec. 2.1 names fast approximate
//    anti-aliasing among its compute passes; the method is Lottes' FXAA,
//    2009).  Every step is a threshold decision, so this one is float32 with
//    the operation order written out (orc_fxaa), matching the product's
//    decisions exactly.
//
// Compile with -O2 -ffp-contract=off -frounding-math (no fast-math).

#include <algorithm>
#include <atomic>
#include <cfenv>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <thread>
#include <vector>

namespace {

// --------------------------------------------------------------------------
// LBVH steps in float32 (bit-exact reference)
// --------------------------------------------------------------------------

inline int clz64(uint64_t x) { return x ? __builtin_clzll(x) : 64; }
inline int clz32(uint32_t x) { return x ? __builtin_clz(x) : 32; }

uint64_t interleave3(uint64_t x, uint64_t y, uint64_t z, int bits) {
    // bit 3i+2 = x_i, 3i+1 = y_i, 3i = z_i
    uint64_t code = 0;
    for (int i = 0; i < bits; ++i) {
        code |= ((x >> i) & 1ull) << (3 * i + 2);
        code |= ((y >> i) & 1ull) << (3 * i + 1);
        code |= ((z >> i) & 1ull) << (3 * i);
    }
    return code;
}

// Augmented common-prefix length of sorted keys i and j (Karras 2012, Sec. 4):
// -1 outside [0,n); for equal keys the indices extend the key.
int delta(const uint64_t* k, int64_t n, int64_t i, int64_t j) {
    if (j < 0 || j >= n) return -1;
    if (k[i] != k[j]) return clz64(k[i] ^ k[j]);
    return 64 + clz32((uint32_t)i ^ (uint32_t)j);
}

// --------------------------------------------------------------------------
// float64 geometry
// --------------------------------------------------------------------------

struct V3 {
    double x, y, z;
    double operator[](int i) const { return i == 0 ? x : (i == 1 ? y : z); }
};
inline V3 operator+(V3 a, V3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 operator-(V3 a, V3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 operator*(double s, V3 a) { return {s * a.x, s * a.y, s * a.z}; }
inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
inline V3 cross(V3 a, V3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }
inline double norm(V3 a) { return std::sqrt(dot(a, a)); }
inline V3 normalize(V3 a) { return (1.0 / norm(a)) * a; }
inline double amax(V3 a) { return std::max(std::fabs(a.x), std::max(std::fabs(a.y), std::fabs(a.z))); }

struct Box {
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    void grow(V3 p) {
        for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], p[a]); hi[a] = std::max(hi[a], p[a]); }
    }
    void grow(const Box& b) {
        for (int a = 0; a < 3; ++a) { lo[a] = std::min(lo[a], b.lo[a]); hi[a] = std::max(hi[a], b.hi[a]); }
    }
};

// Slab test of a box widened by `pad` on every side against the ray interval
// [t0, t1]; returns the entry distance or +inf.
double box_hit(const Box& b, double pad, V3 o, V3 d, double t0, double t1) {
    double tn = t0, tf = t1;
    for (int a = 0; a < 3; ++a) {
        double lo = b.lo[a] - pad, hi = b.hi[a] + pad;
        if (d[a] == 0.0) {
            if (o[a] < lo || o[a] > hi) return INFINITY;
            continue;
        }
        double inv = 1.0 / d[a];
        double ta = (lo - o[a]) * inv, tb = (hi - o[a]) * inv;
        if (ta > tb) std::swap(ta, tb);
        tn = std::max(tn, ta);
        tf = std::min(tf, tb);
    }
    // relative slack for float64 rounding of the slab distances
    if (tn <= tf * (1.0 + 1e-12) + 1e-300) return tn;
    return INFINITY;
}

// Object-median BVH over item boxes (leaves of <= 4 items).
struct Bvh {
    struct Node { Box box; int left = -1, right = -1, first = 0, count = 0; };
    std::vector<Node> nodes;
    std::vector<uint32_t> items;

    void build(const std::vector<Box>& boxes) {
        items.resize(boxes.size());
        for (size_t i = 0; i < boxes.size(); ++i) items[i] = (uint32_t)i;
        nodes.clear();
        nodes.reserve(2 * boxes.size() + 1);
        if (boxes.empty()) return;
        build_rec(boxes, 0, (int)boxes.size());
    }
    int build_rec(const std::vector<Box>& boxes, int first, int count) {
        int id = (int)nodes.size();
        nodes.emplace_back();
        Box b, cb;
        for (int i = first; i < first + count; ++i) {
            b.grow(boxes[items[i]]);
            const Box& x = boxes[items[i]];
            cb.grow(V3{(x.lo[0] + x.hi[0]) * 0.5, (x.lo[1] + x.hi[1]) * 0.5, (x.lo[2] + x.hi[2]) * 0.5});
        }
        nodes[id].box = b;
        if (count <= 4) { nodes[id].first = first; nodes[id].count = count; return id; }
        int axis = 0;
        for (int a = 1; a < 3; ++a)
            if (cb.hi[a] - cb.lo[a] > cb.hi[axis] - cb.lo[axis]) axis = a;
        int mid = first + count / 2;
        std::nth_element(items.begin() + first, items.begin() + mid, items.begin() + first + count,
                         [&](uint32_t p, uint32_t q) {
                             double cp = boxes[p].lo[axis] + boxes[p].hi[axis];
                             double cq = boxes[q].lo[axis] + boxes[q].hi[axis];
                             return cp < cq || (cp == cq && p < q);
                         });
        int l = build_rec(boxes, first, mid - first);
        int r = build_rec(boxes, mid, first + count - mid);
        nodes[id].left = l;
        nodes[id].right = r;
        return id;
    }
};

struct Mesh {
    std::vector<V3> v;            // vertices (exact float32 values in float64)
    std::vector<uint32_t> idx;    // 3 per triangle
    std::vector<double> inv_h;    // 3 per triangle: 1/altitude opposite vertex i (0 if degenerate)
    std::vector<V3> ng;           // unit geometric normal (0 if degenerate)
    Bvh bvh;
    Box box;
    double vmax = 0;
};

struct Instance {
    double M[12];      // object -> world (row-major 3x4)
    double Minv[12];   // world -> object
    uint32_t mesh;
    uint32_t material;
    Box wbox;          // world box (float64 transform of the 8 object-box corners)
};

struct Scene {
    std::vector<Mesh> meshes;
    std::vector<Instance> inst;
    Bvh tlas;
    // shading
    std::vector<uint32_t> mat_type;
    std::vector<V3> mat_albedo;
    std::vector<double> mat_ior;
    std::vector<V3> light_pos, light_I;
    V3 background{0.2, 0.3, 0.5};
    double ambient = 0.1;
};

constexpr double EPS32 = 5.9604644775390625e-08;  // 2^-24, float32 unit roundoff
constexpr double kGrazeInv = 256.0;                // |cos| below 1/256 counts as grazing

inline V3 xform_point(const double* m, V3 p) {
    return {m[0] * p.x + m[1] * p.y + m[2] * p.z + m[3], m[4] * p.x + m[5] * p.y + m[6] * p.z + m[7],
            m[8] * p.x + m[9] * p.y + m[10] * p.z + m[11]};
}
inline V3 xform_dir(const double* m, V3 d) {
    return {m[0] * d.x + m[1] * d.y + m[2] * d.z, m[4] * d.x + m[5] * d.y + m[6] * d.z,
            m[8] * d.x + m[9] * d.y + m[10] * d.z};
}

// Inverse of a 3x4 affine map [A | t] in float64: A^-1 = adj(A)/det, t' = -A^-1 t.
bool invert34(const double* m, double* r, double* det_out) {
    double a = m[0], b = m[1], c = m[2], d = m[4], e = m[5], f = m[6], g = m[8], h = m[9], i = m[10];
    double A = e * i - f * h, B = -(d * i - f * g), C = d * h - e * g;
    double det = a * A + b * B + c * C;
    if (det_out) *det_out = det;
    if (det == 0.0) return false;
    double id = 1.0 / det;
    double inv[9] = {A * id, -(b * i - c * h) * id, (b * f - c * e) * id,
                     B * id, (a * i - c * g) * id, -(a * f - c * d) * id,
                     C * id, -(a * h - b * g) * id, (a * e - b * d) * id};
    for (int row = 0; row < 3; ++row) {
        r[4 * row + 0] = inv[3 * row + 0];
        r[4 * row + 1] = inv[3 * row + 1];
        r[4 * row + 2] = inv[3 * row + 2];
        r[4 * row + 3] = -(inv[3 * row + 0] * m[3] + inv[3 * row + 1] * m[7] + inv[3 * row + 2] * m[11]);
    }
    return true;
}

// Watertight ray/triangle test (Woop, Benthin, Wald, JCGT 2013) in float64.
// Returns the edge functions U (weight of v0), V (v1), W (v2), their sum det
// and the scaled distance T, so that t = T/det and barycentrics = (U,V,W)/det.
struct WT { double U, V, W, det, T; };
struct RayPre { int kx, ky, kz; double Sx, Sy, Sz; };

RayPre precompute(V3 d) {
    RayPre p;
    double ax = std::fabs(d.x), ay = std::fabs(d.y), az = std::fabs(d.z);
    p.kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    p.kx = (p.kz + 1) % 3;
    p.ky = (p.kx + 1) % 3;
    if (d[p.kz] < 0) std::swap(p.kx, p.ky);
    p.Sx = d[p.kx] / d[p.kz];
    p.Sy = d[p.ky] / d[p.kz];
    p.Sz = 1.0 / d[p.kz];
    return p;
}

WT watertight(const RayPre& p, V3 o, V3 v0, V3 v1, V3 v2) {
    V3 A = v0 - o, B = v1 - o, C = v2 - o;
    double Ax = A[p.kx] - p.Sx * A[p.kz], Ay = A[p.ky] - p.Sy * A[p.kz];
    double Bx = B[p.kx] - p.Sx * B[p.kz], By = B[p.ky] - p.Sy * B[p.kz];
    double Cx = C[p.kx] - p.Sx * C[p.kz], Cy = C[p.ky] - p.Sy * C[p.kz];
    WT w;
    w.U = Cx * By - Cy * Bx;
    w.V = Ax * Cy - Ay * Cx;
    w.W = Bx * Ay - By * Ax;
    w.det = w.U + w.V + w.W;
    w.T = w.U * (p.Sz * A[p.kz]) + w.V * (p.Sz * B[p.kz]) + w.W * (p.Sz * C[p.kz]);
    return w;
}

// ---- ray query with the ambiguity classification --------------------------
//
// For each triangle the exact (float64) test gives the ray/plane point's
// barycentrics b_i and distance t.  The float32 pipeline computes the same
// point with an absolute position error of at most eta (object-space units):
//   eta = kappa * 2^-24 * (|Minv||o| + |m| + t |Minv||d| + max|v|),
// i.e. a few roundings of the largest magnitudes that enter the transformed
// ray and the sheared vertices.  Moving the ray by eta moves its plane point
// by up to eta_p = eta / |cos| (cos between the ray and the triangle normal;
// capped at |cos| = 1/256, below which the hit counts as grazing).  A triangle is
//   strict : the exact test accepts it (b_i >= 0, det != 0, t in range);
//   outer  : the point lies within eta_p of the triangle (b_i h_i >= -eta_p);
//   inner  : strict, not grazing, and at least eta_p inside every edge.
// A closest-hit ray is ambiguous when the float32 answer may differ from the
// exact one: the exact winner is not inner, another outer candidate lies
// within the distance tolerance of the winner, or there is no winner but an
// outer candidate exists.  An any-hit ray is ambiguous when the outer and the
// inner tests disagree on whether the segment is blocked.

struct Cand { double t; uint32_t inst, prim; bool strict, inner; double u, v, tau, bary_tol; };

struct QueryOut {
    bool hit = false;
    uint32_t inst = 0xFFFFFFFFu, prim = 0xFFFFFFFFu;
    double t = INFINITY, u = 0, v = 0;
    bool ambiguous = false;
    double tol_t = 0, tol_b = 0;
    V3 n_world{0, 0, 0};  // unit geometric normal of the winner, world space (un-flipped)
};

struct Query {
    const Scene& S;
    double kappa;
    double rel_t;  // relative distance tolerance (near ties, interval ends)
    Query(const Scene& s, double k, double r) : S(s), kappa(k), rel_t(r) {}

    // test every triangle of instance k (brute) or its BLAS
    template <class F>
    void visit_instance(uint32_t k, V3 o, V3 d, double t0, double t1_cull, bool brute, F&& on_tri) const {
        const Instance& I = S.inst[k];
        const Mesh& m = S.meshes[I.mesh];
        V3 oo = xform_point(I.Minv, o), dd = xform_dir(I.Minv, d);
        // error scale of the object-space ray (see above)
        double E0 = 0, E1 = 0;
        for (int r = 0; r < 3; ++r) {
            double s0 = std::fabs(I.Minv[4 * r + 3]), s1 = 0;
            for (int c = 0; c < 3; ++c) {
                s0 += std::fabs(I.Minv[4 * r + c]) * std::fabs(o[c]);
                s1 += std::fabs(I.Minv[4 * r + c]) * std::fabs(d[c]);
            }
            E0 = std::max(E0, s0);
            E1 = std::max(E1, s1);
        }
        RayPre pre = precompute(dd);
        double dn = norm(dd);
        auto test = [&](uint32_t prim) {
            V3 v0 = m.v[m.idx[3 * prim]], v1 = m.v[m.idx[3 * prim + 1]], v2 = m.v[m.idx[3 * prim + 2]];
            if (m.inv_h[3 * prim] == 0.0) return;  // zero-area triangle: never hit
            WT w = watertight(pre, oo, v0, v1, v2);
            if (w.det == 0.0) return;
            double t = w.T / w.det;
            double b0 = w.U / w.det, b1 = w.V / w.det, b2 = w.W / w.det;
            double eta = kappa * EPS32 * (E0 + std::fabs(t) * E1 + m.vmax);
            double e0 = b0 / m.inv_h[3 * prim], e1 = b1 / m.inv_h[3 * prim + 1], e2 = b2 / m.inv_h[3 * prim + 2];
            double cosv = std::fabs(dot(m.ng[prim], dd)) / dn;
            // an offset eta of the ray moves its plane point by up to eta/|cos|
            // within the plane (along the ray by eta/(|cos| |d|) in t); below
            // |cos| = 1/kGrazeInv the band stops growing and the hit is never
            // "inner" (so a grazing winner is always ambiguous)
            bool grazing = cosv * kGrazeInv < 1.0;
            double eta_p = eta * (grazing ? kGrazeInv : 1.0 / cosv);
            double tau = rel_t * std::fabs(t) + eta_p / dn;
            bool outer = e0 >= -eta_p && e1 >= -eta_p && e2 >= -eta_p;
            if (!outer) return;
            bool inside = (w.U >= 0 && w.V >= 0 && w.W >= 0) || (w.U <= 0 && w.V <= 0 && w.W <= 0);
            bool strict = inside && t >= t0 && t <= t1_cull;  // caller re-checks against tmax
            bool inner = inside && !grazing && e0 >= eta_p && e1 >= eta_p && e2 >= eta_p;
            double hmin_inv = std::max(m.inv_h[3 * prim], std::max(m.inv_h[3 * prim + 1], m.inv_h[3 * prim + 2]));
            on_tri(Cand{t, k, prim, strict, inner, b1, b2, tau, eta_p * hmin_inv}, eta);
        };
        if (brute) {
            uint32_t nt = (uint32_t)(m.idx.size() / 3);
            for (uint32_t p = 0; p < nt; ++p) test(p);
            return;
        }
        if (m.bvh.nodes.empty()) return;
        // BLAS boxes are widened by the largest eta any hit inside this instance can have
        double tup = INFINITY;
        {
            V3 c{(m.box.lo[0] + m.box.hi[0]) / 2, (m.box.lo[1] + m.box.hi[1]) / 2, (m.box.lo[2] + m.box.hi[2]) / 2};
            V3 ext{m.box.hi[0] - c.x, m.box.hi[1] - c.y, m.box.hi[2] - c.z};
            tup = (norm(oo - c) + norm(ext)) / dn;
        }
        // a candidate's plane point lies within eta * kGrazeInv of its triangle
        double pad = kGrazeInv * kappa * EPS32 * (E0 + tup * E1 + m.vmax) * 2 + 1e-12 * (1 + m.vmax);
        double tlo = t0 - 1e-3 * (amax(o) + 1.0);
        int stack[256];
        int sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            int ni = stack[--sp];
            const Bvh::Node& nd = m.bvh.nodes[ni];
            if (box_hit(nd.box, pad, oo, dd, tlo, cull_limit()) == INFINITY) continue;
            if (nd.left < 0) {
                for (int i = nd.first; i < nd.first + nd.count; ++i) test(m.bvh.items[i]);
            } else {
                stack[sp++] = nd.left;
                stack[sp++] = nd.right;
            }
            if (done) return;
        }
        (void)t1_cull;
    }

    // mutable traversal state
    mutable double cull = INFINITY;
    mutable bool done = false;
    double cull_limit() const { return cull; }

    template <class F>
    void visit_all(V3 o, V3 d, double t0, double t1, bool brute, F&& on_tri) const {
        if (brute || S.tlas.nodes.empty()) {
            for (uint32_t k = 0; k < S.inst.size(); ++k) {
                visit_instance(k, o, d, t0, t1, brute, on_tri);
                if (done) return;
            }
            return;
        }
        double pad = 1e-3 * (amax(o) + 1.0);
        double tlo = t0 - 1e-3 * (amax(o) + 1.0);
        int stack[256];
        int sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            int ni = stack[--sp];
            const Bvh::Node& nd = S.tlas.nodes[ni];
            double ext = 0;
            for (int a = 0; a < 3; ++a) ext = std::max(ext, nd.box.hi[a] - nd.box.lo[a]);
            if (box_hit(nd.box, pad + 1e-3 * ext, o, d, tlo, cull) == INFINITY) continue;
            if (nd.left < 0) {
                for (int i = nd.first; i < nd.first + nd.count; ++i) {
                    visit_instance(S.tlas.items[i], o, d, t0, t1, false, on_tri);
                    if (done) return;
                }
            } else {
                stack[sp++] = nd.left;
                stack[sp++] = nd.right;
            }
        }
    }

    QueryOut closest(V3 o, V3 d, double tmin, double tmax, bool brute) const {
        std::vector<Cand> cands;
        Cand best{INFINITY, 0xFFFFFFFFu, 0xFFFFFFFFu, false, false, 0, 0, 0, 0};
        bool have = false;
        cull = std::isinf(tmax) ? INFINITY : tmax * (1 + 1e-3) + 1e-3;
        done = false;
        double scale = amax(o) + 1.0;
        // the window searched for candidates is the one the BVH traversal keeps
        const double t_lo = tmin - 1e-3 * (amax(o) + 1.0);
        visit_all(o, d, tmin, tmax, brute, [&](const Cand& c, double) {
            if (c.t < tmin - c.tau || c.t > tmax + c.tau || c.t < t_lo || c.t > cull) return;
            cands.push_back(c);
            if (c.strict && c.t <= tmax) {
                // the nearest hit, with distances compared as float32 values
                // (the precision the hit records carry): equal float32 t is a
                // tie, decided by the smaller instance, then the smaller prim
                const float ct = (float)c.t, bt = (float)best.t;
                bool better = !have || ct < bt ||
                              (ct == bt && (c.inst < best.inst || (c.inst == best.inst && c.prim < best.prim)));
                if (better) {
                    best = c;
                    have = true;
                    // monotone in best.t, so the final value does not depend on visit order
                    cull = std::min(cull, best.t * (1 + 1e-3) + 1e-3 * scale);
                }
            }
        });
        QueryOut q;
        if (have) {
            q.hit = true;
            q.inst = best.inst;
            q.prim = best.prim;
            q.t = best.t;
            q.u = best.u;
            q.v = best.v;
            q.tol_t = best.tau;
            q.tol_b = best.bary_tol + rel_t;
            bool amb = !best.inner || best.t - best.tau < tmin || best.t + best.tau > tmax;
            // candidates beyond the final cull distance are ignored, so that the
            // BVH and the brute-force traversal see the same candidate set
            for (const Cand& c : cands) {
                if (c.inst == best.inst && c.prim == best.prim) continue;
                if (c.t > cull) continue;
                if (c.t <= best.t + best.tau + c.tau) { amb = true; break; }
            }
            q.ambiguous = amb;
            const Instance& I = S.inst[best.inst];
            const Mesh& m = S.meshes[I.mesh];
            V3 n = m.ng[best.prim];
            // world normal = Minv^T n
            V3 nw{I.Minv[0] * n.x + I.Minv[4] * n.y + I.Minv[8] * n.z, I.Minv[1] * n.x + I.Minv[5] * n.y + I.Minv[9] * n.z,
                  I.Minv[2] * n.x + I.Minv[6] * n.y + I.Minv[10] * n.z};
            q.n_world = normalize(nw);
        } else {
            q.ambiguous = !cands.empty();
        }
        return q;
    }

    // any-hit: returns occluded, sets ambiguous when outer and inner tests disagree
    bool any(V3 o, V3 d, double tmin, double tmax, bool brute, bool* ambiguous) const {
        bool outer_blocked = false, inner_blocked = false, strict_blocked = false;
        cull = std::isinf(tmax) ? INFINITY : tmax * (1 + 1e-3) + 1e-3;
        done = false;
        const double t_lo = tmin - 1e-3 * (amax(o) + 1.0);
        visit_all(o, d, tmin, tmax, brute, [&](const Cand& c, double) {
            if (c.t < t_lo || c.t > cull) return;
            if (c.t >= tmin - c.tau && c.t <= tmax + c.tau) outer_blocked = true;
            if (c.strict && c.t >= tmin && c.t <= tmax) strict_blocked = true;
            if (c.inner && c.t >= tmin + c.tau && c.t <= tmax - c.tau) {
                inner_blocked = true;
                done = true;
            }
        });
        if (inner_blocked) strict_blocked = true;
        *ambiguous = outer_blocked != inner_blocked;
        return strict_blocked;
    }
};

// ---- Whitted shading (float64) ---------------------------------------------

// Mirror direction of unit d about the unit normal nf: d - 2 (d.nf) nf.
V3 reflect_dir(V3 d, V3 nf) { return normalize(d - (2.0 * dot(d, nf)) * nf); }

// Refraction through a surface of index ior (the other side has index 1).
// nf faces against d; `entering` is true when d travels into the material.
// Snell: eta = n1/n2, cos_i = -d.nf, k = 1 - eta^2 (1 - cos_i^2); k < 0 is
// total internal reflection (returns false).  Otherwise T = eta d +
// (eta cos_i - sqrt k) nf, and R is Schlick's Fresnel approximation
// R0 + (1-R0)(1-c)^5 with R0 = ((1-ior)/(1+ior))^2 and c the cosine on the
// vacuum side (cos_i when entering, sqrt k when leaving).
bool refract_dir(V3 d, V3 nf, bool entering, double ior, V3* T, double* R) {
    double eta = entering ? 1.0 / ior : ior;
    double ci = -dot(d, nf);
    double k = 1.0 - eta * eta * (1.0 - ci * ci);
    if (k < 0) return false;
    double sk = std::sqrt(k);
    *T = normalize(eta * d + (eta * ci - sk) * nf);
    double R0 = ((1 - ior) / (1 + ior)) * ((1 - ior) / (1 + ior));
    double c = entering ? ci : sk;
    *R = R0 + (1 - R0) * std::pow(1 - c, 5);
    return true;
}

struct Shade {
    const Scene& S;
    const Query& Q;
    int max_depth;
    uint64_t* counts;  // [closest, shadow]
    bool amb = false;

    V3 trace(V3 o, V3 d, int depth, bool* hit_out) {
        counts[0]++;
        QueryOut h = Q.closest(o, d, 0.0, INFINITY, false);
        if (h.ambiguous) amb = true;
        if (hit_out) *hit_out = h.hit;
        if (!h.hit) return S.background;
        const Instance& I = S.inst[h.inst];
        uint32_t mi = I.material;
        V3 p = o + h.t * d;
        V3 n = h.n_world;
        bool entering = dot(d, n) < 0;
        V3 nf = entering ? n : (-1.0) * n;
        double eps = 1e-4 * std::max(1.0, amax(p));
        uint32_t type = S.mat_type[mi];
        V3 a = S.mat_albedo[mi];
        if (type == 0) {  // diffuse
            V3 L = S.ambient * a;
            V3 os = p + eps * nf;
            for (size_t l = 0; l < S.light_pos.size(); ++l) {
                V3 lv = S.light_pos[l] - os;
                double dist = norm(lv);
                V3 ld = (1.0 / dist) * lv;
                double c = dot(nf, ld);
                if (c <= 0) continue;
                counts[1]++;
                bool sa = false;
                bool occ = Q.any(os, ld, 0.0, dist - eps, false, &sa);
                if (sa) amb = true;
                if (!occ) {
                    V3 I_l = S.light_I[l];
                    L = L + V3{a.x * I_l.x * c, a.y * I_l.y * c, a.z * I_l.z * c};
                }
            }
            return L;
        }
        if (depth >= max_depth) return {0, 0, 0};
        V3 r = reflect_dir(d, nf);
        if (type == 1) {  // mirror
            V3 Lr = trace(p + eps * nf, r, depth + 1, nullptr);
            return {a.x * Lr.x, a.y * Lr.y, a.z * Lr.z};
        }
        // glass
        V3 T;
        double R;
        if (!refract_dir(d, nf, entering, S.mat_ior[mi], &T, &R))
            return trace(p + eps * nf, r, depth + 1, nullptr);  // total internal reflection
        V3 Lr = trace(p + eps * nf, r, depth + 1, nullptr);
        V3 Lt = trace(p - eps * nf, T, depth + 1, nullptr);
        return R * Lr + (1 - R) * Lt;
    }
};

V3 camera_dir(const float* cam, uint32_t w, uint32_t h, uint32_t x, uint32_t y) {
    V3 eye{cam[0], cam[1], cam[2]}, tgt{cam[3], cam[4], cam[5]}, up{cam[6], cam[7], cam[8]};
    double th = std::tan(0.5 * (double)cam[9] * M_PI / 180.0);
    double aspect = (double)w / (double)h;
    V3 F = normalize(tgt - eye);
    V3 R = normalize(cross(F, up));
    V3 U = cross(R, F);
    double px = (2.0 * (x + 0.5) / w - 1.0) * aspect * th;
    double py = (1.0 - 2.0 * (y + 0.5) / h) * th;
    return normalize(px * R + py * U + F);
}

template <class F>
void parallel_for(int64_t n, int nthreads, F&& f) {
    if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
    if (nthreads == 1 || n < 64) {
        for (int64_t i = 0; i < n; ++i) f(i);
        return;
    }
    std::atomic<int64_t> next{0};
    const int64_t chunk = 64;
    std::vector<std::thread> th;
    for (int t = 0; t < nthreads; ++t)
        th.emplace_back([&]() {
            for (;;) {
                int64_t b = next.fetch_add(chunk);
                if (b >= n) break;
                int64_t e = std::min(n, b + chunk);
                for (int64_t i = b; i < e; ++i) f(i);
            }
        });
    for (auto& t : th) t.join();
}

}  // namespace

extern "C" {

// ---- LBVH reference steps ----------------------------------------------------

// Per-triangle object box (exact float32 min/max of the three vertices).
// lohi[6*i] = {lo.x, lo.y, lo.z, hi.x, hi.y, hi.z}.
int orc_tri_bounds(const float* vtx, uint32_t nv, const uint32_t* idx, uint32_t nt, float* lohi) {
    for (uint32_t i = 0; i < nt; ++i) {
        for (int a = 0; a < 3; ++a) {
            float lo = INFINITY, hi = -INFINITY;
            for (int c = 0; c < 3; ++c) {
                uint32_t vi = idx[3 * i + c];
                if (vi >= nv) return -1;
                float x = vtx[3 * vi + a];
                lo = std::min(lo, x);
                hi = std::max(hi, x);
            }
            lohi[6 * i + a] = lo;
            lohi[6 * i + 3 + a] = hi;
        }
    }
    return 0;
}

// Morton code of each box centroid.  c = (lo+hi)*0.5f; per axis
// s = 2^b / (cmax-cmin) and q = clamp(floor((c-cmin)*s), 0, 2^b-1), q = 0 on a
// degenerate axis; bits interleaved x (MSB), y, z.  All float32, fixed order.
int orc_morton(const float* lohi, uint32_t n, int bits, uint64_t* codes, float* cbounds) {
    float cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
    std::vector<float> c(3 * (size_t)n);
    for (uint32_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            volatile float s = lohi[6 * i + a] + lohi[6 * i + 3 + a];
            float ca = s * 0.5f;
            c[3 * (size_t)i + a] = ca;
            cmin[a] = std::min(cmin[a], ca);
            cmax[a] = std::max(cmax[a], ca);
        }
    // one scale 2^bits / (largest centroid extent) for all three axes
    const float full = (float)(1u << bits);
    const float qmax = (float)((1u << bits) - 1u);
    float ext = 0.0f;
    for (int a = 0; a < 3; ++a) {
        volatile float e = cmax[a] - cmin[a];
        if (cmax[a] > cmin[a] && e > ext) ext = e;
    }
    volatile float scale = ext > 0.0f ? full / ext : 0.0f;
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t q[3];
        for (int a = 0; a < 3; ++a) {
            if (!(cmax[a] > cmin[a])) { q[a] = 0; continue; }
            volatile float off = c[3 * (size_t)i + a] - cmin[a];
            volatile float f = off * scale;
            float fl = std::floor((float)f);
            fl = std::min(std::max(fl, 0.0f), qmax);
            q[a] = (uint64_t)fl;
        }
        codes[i] = interleave3(q[0], q[1], q[2], bits);
    }
    if (cbounds) {
        for (int a = 0; a < 3; ++a) { cbounds[a] = cmin[a]; cbounds[3 + a] = cmax[a]; }
    }
    return 0;
}

// Stable sort: perm lists the indices of `keys` in (key, index) order.
int orc_stable_sort(const uint64_t* keys, uint32_t n, uint32_t* perm) {
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    std::stable_sort(perm, perm + n, [&](uint32_t a, uint32_t b) { return keys[a] < keys[b]; });
    return 0;
}

// Binary radix tree over sorted keys, built top-down.  Internal node ids follow
// Karras 2012: the root is node 0 and covers [0, n-1]; a node covering
// [first, last] splits at gamma = max{ i in [first, last-1] : delta(first, i) >
// delta(first, last) }; its left child is leaf `first` if gamma == first, else
// internal node gamma; its right child is leaf `last` if gamma+1 == last, else
// internal node gamma+1.  Outputs per internal node: first, last, split.
int orc_karras(const uint64_t* k, uint32_t n, int32_t* first, int32_t* last, int32_t* split) {
    if (n < 2) return 0;
    std::vector<int64_t> st;
    st.push_back(0);
    std::vector<std::pair<int64_t, int64_t>> range(n - 1, {-1, -1});
    range[0] = {0, (int64_t)n - 1};
    while (!st.empty()) {
        int64_t id = st.back();
        st.pop_back();
        int64_t f = range[id].first, l = range[id].second;
        int dn = delta(k, n, f, l);
        int64_t g = f;
        while (g + 1 <= l - 1 && delta(k, n, f, g + 1) > dn) ++g;
        first[id] = (int32_t)f;
        last[id] = (int32_t)l;
        split[id] = (int32_t)g;
        if (g != f) { range[g] = {f, g}; st.push_back(g); }
        if (g + 1 != l) { range[g + 1] = {g + 1, l}; st.push_back(g + 1); }
    }
    return 0;
}

// Binned surface-area-heuristic hierarchy (the BLAS build for trace speed;
// the paper's framework leaves acceleration structures to the Vulkan driver,
// so this build is a choice of the implementation, written out here in its
// plain definition).  The leaves start in Morton order.  A range of c leaves
// at depth `level` whose root is internal node d:
//   * c <= 2 or level >= 40: the Karras hierarchy of the range's own keys
//     (local indices), its node j numbered d + j, its leaf j numbered b + j;
//   * otherwise, per axis, 16 bins of the centroids c = 0.5 (lo + hi) over the
//     range's centroid bounds: bin = floor((c - cmin) * s), s = 16 / (cmax -
//     cmin) (capped at 3e38; 0 for a point), clamped to 0..15 (NaN to 0); the
//     boundary of least A(left) n(left) + A(right) n(right), A the half area
//     dx dy + dy dz + dz dx of the union box, taken over axes 0, 1, 2 and
//     boundaries 1..15 in that order, the first of equal costs kept; when
//     every side split leaves one side empty, the range is halved by
//     position.  The range is partitioned stably (left leaves first, each
//     side in its previous order); node d's children are node d + 1 (or leaf
//     b when one leaf) and node d + n(left) (or leaf b + n(left)).
// Every operation is float32 as written (no contraction).  Outputs: perm_out,
// the triangle of each leaf, and child, two per internal node (bit 31: leaf).
int orc_sah_build(const float* lohi, uint32_t n, const uint64_t* sorted_keys, const uint32_t* perm_in,
                  uint32_t* perm_out, uint32_t* child) {
    const uint32_t kLeafBit = 0x80000000u;
    std::vector<uint32_t> prim(perm_in, perm_in + n);
    std::vector<uint64_t> key(sorted_keys, sorted_keys + n);
    struct Range {
        uint32_t b, c, d, level;
    };
    std::vector<Range> todo;
    if (n >= 2) todo.push_back({0u, n, 0u, 0u});
    auto centroid = [&](uint32_t t, int a) { return 0.5f * (lohi[6 * (size_t)t + a] + lohi[6 * (size_t)t + 3 + a]); };
    auto half_area = [](const float* lo, const float* hi) {
        const float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
        return (dx * dy + dy * dz) + dz * dx;
    };
    while (!todo.empty()) {
        const Range R = todo.back();
        todo.pop_back();
        if (R.c <= 2 || R.level >= 40) {
            std::vector<int32_t> f(R.c - 1), l(R.c - 1), sp(R.c - 1);
            orc_karras(key.data() + R.b, R.c, f.data(), l.data(), sp.data());
            for (uint32_t j = 0; j + 1 < R.c; ++j) {
                const uint32_t g = (uint32_t)sp[j];
                child[2 * (size_t)(R.d + j)] = (uint32_t)f[j] == g ? (kLeafBit | (R.b + g)) : R.d + g;
                child[2 * (size_t)(R.d + j) + 1] = (uint32_t)l[j] == g + 1 ? (kLeafBit | (R.b + g + 1)) : R.d + g + 1;
            }
            continue;
        }
        float cmin[3] = {INFINITY, INFINITY, INFINITY}, cmax[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (uint32_t p = R.b; p < R.b + R.c; ++p)
            for (int a = 0; a < 3; ++a) {
                cmin[a] = std::min(cmin[a], centroid(prim[p], a));
                cmax[a] = std::max(cmax[a], centroid(prim[p], a));
            }
        float scale[3];
        for (int a = 0; a < 3; ++a) {
            const float ext = cmax[a] - cmin[a];
            scale[a] = ext > 0.0f ? std::min(16.0f / ext, 3.0e38f) : 0.0f;
        }
        auto bin = [&](uint32_t t, int a) {
            const float v = (centroid(t, a) - cmin[a]) * scale[a];
            if (!(v >= 0.0f)) return 0;
            return v < 16.0f ? (int)v : 15;
        };
        uint32_t cnt[3][16] = {};
        float blo[3][16][3], bhi[3][16][3];
        for (int a = 0; a < 3; ++a)
            for (int k = 0; k < 16; ++k)
                for (int q = 0; q < 3; ++q) {
                    blo[a][k][q] = INFINITY;
                    bhi[a][k][q] = -INFINITY;
                }
        for (uint32_t p = R.b; p < R.b + R.c; ++p)
            for (int a = 0; a < 3; ++a) {
                const int k = bin(prim[p], a);
                ++cnt[a][k];
                for (int q = 0; q < 3; ++q) {
                    blo[a][k][q] = std::min(blo[a][k][q], lohi[6 * (size_t)prim[p] + q]);
                    bhi[a][k][q] = std::max(bhi[a][k][q], lohi[6 * (size_t)prim[p] + 3 + q]);
                }
            }
        float best = INFINITY;
        int best_axis = -1, best_split = 0;
        uint32_t nl = R.c / 2;
        for (int a = 0; a < 3; ++a)
            for (int s = 1; s < 16; ++s) {
                float llo[3] = {INFINITY, INFINITY, INFINITY}, lhi[3] = {-INFINITY, -INFINITY, -INFINITY};
                float rlo[3] = {INFINITY, INFINITY, INFINITY}, rhi[3] = {-INFINITY, -INFINITY, -INFINITY};
                uint32_t cl = 0, cr = 0;
                for (int k = 0; k < 16; ++k) {
                    float* lo = k < s ? llo : rlo;
                    float* hi = k < s ? lhi : rhi;
                    (k < s ? cl : cr) += cnt[a][k];
                    for (int q = 0; q < 3; ++q) {
                        lo[q] = std::min(lo[q], blo[a][k][q]);
                        hi[q] = std::max(hi[q], bhi[a][k][q]);
                    }
                }
                if (cl == 0 || cr == 0) continue;
                const float cost = half_area(llo, lhi) * (float)cl + half_area(rlo, rhi) * (float)cr;
                if (cost < best) {
                    best = cost;
                    best_axis = a;
                    best_split = s;
                    nl = cl;
                }
            }
        std::vector<uint32_t> lp, rp;
        std::vector<uint64_t> lk, rk;
        for (uint32_t p = R.b; p < R.b + R.c; ++p) {
            const bool left = best_axis < 0 ? (p - R.b < nl) : (bin(prim[p], best_axis) < best_split);
            (left ? lp : rp).push_back(prim[p]);
            (left ? lk : rk).push_back(key[p]);
        }
        std::copy(lp.begin(), lp.end(), prim.begin() + R.b);
        std::copy(rp.begin(), rp.end(), prim.begin() + R.b + nl);
        std::copy(lk.begin(), lk.end(), key.begin() + R.b);
        std::copy(rk.begin(), rk.end(), key.begin() + R.b + nl);
        const uint32_t nr = R.c - nl;
        child[2 * (size_t)R.d] = nl == 1 ? (kLeafBit | R.b) : R.d + 1;
        child[2 * (size_t)R.d + 1] = nr == 1 ? (kLeafBit | (R.b + nl)) : R.d + nl;
        if (nl >= 2) todo.push_back({R.b, nl, R.d + 1, R.level + 1});
        if (nr >= 2) todo.push_back({R.b + nl, nr, R.d + nl, R.level + 1});
    }
    std::copy(prim.begin(), prim.end(), perm_out);
    return 0;
}

// Box of every internal node = union of the (sorted) leaf boxes in its range.
int orc_range_boxes(const float* lohi_sorted, uint32_t n, const int32_t* first, const int32_t* last, float* boxes) {
    for (uint32_t i = 0; i + 1 < n; ++i) {
        float b[6] = {INFINITY, INFINITY, INFINITY, -INFINITY, -INFINITY, -INFINITY};
        for (int32_t j = first[i]; j <= last[i]; ++j)
            for (int a = 0; a < 3; ++a) {
                b[a] = std::min(b[a], lohi_sorted[6 * (size_t)j + a]);
                b[3 + a] = std::max(b[3 + a], lohi_sorted[6 * (size_t)j + 3 + a]);
            }
        std::memcpy(boxes + 6 * (size_t)i, b, sizeof b);
    }
    return 0;
}

// Per instance: float64 inverse of the object-to-world 3x4 M (returns -2 if
// singular) and the world box of the object box by Arvo's method,
//   lo_i = (((min(M_i0 a_0, M_i0 b_0) + min(M_i1 a_1, M_i1 b_1)) + min(M_i2 a_2, M_i2 b_2)) + t_i)
// with every float32 product and sum rounded toward -inf (hi: max, toward +inf).
// Bound on the squared distance of a mesh's vertices from its root box centre
// c = (lo + hi) * 0.5 (float32): the largest over the vertices of
// (|dx|^2 + |dy|^2) + |dz|^2, every operation rounded upward.
float orc_bound_r2(const float* vtx, uint32_t nv, const float* box) {
    const int old = std::fegetround();
    float c[3];
    for (int i = 0; i < 3; ++i) c[i] = (box[i] + box[3 + i]) * 0.5f;
    std::fesetround(FE_UPWARD);
    volatile float best = 0.0f;
    for (uint32_t v = 0; v < nv; ++v) {
        volatile float e[3];
        for (int i = 0; i < 3; ++i) {
            const float x = vtx[3 * (size_t)v + i];
            e[i] = x >= c[i] ? x - c[i] : c[i] - x;
        }
        volatile float sx = e[0] * e[0], sy = e[1] * e[1], sz = e[2] * e[2];
        volatile float d2 = sx + sy;
        d2 = d2 + sz;
        if (d2 > best) best = d2;
    }
    std::fesetround(old);
    return best;
}

// Instance prep: float64 inverse, and the world box of the instance: Arvo's
// box of the transformed object box, intersected (when obj_r2 is given) with
// the box of the transformed bounding sphere (centre c of the object box,
// radius sqrt(r2)): A c + t -/+ r |row_i(A)|, with outward rounding.
int orc_instance_prep(const float* M, uint32_t n, const float* obj_box, const float* obj_r2, double* Minv,
                      float* wbox) {
    int rc = 0;
    const int old = std::fegetround();
    for (uint32_t k = 0; k < n; ++k) {
        double m[12];
        for (int i = 0; i < 12; ++i) m[i] = M[12 * k + i];
        double det;
        if (!invert34(m, Minv + 12 * (size_t)k, &det)) rc = -2;
        const float* a = obj_box + 6 * (size_t)k;
        for (int i = 0; i < 3; ++i) {
            std::fesetround(FE_DOWNWARD);
            volatile float s = 0.0f;
            for (int j = 0; j < 3; ++j) {
                volatile float p0 = M[12 * k + 4 * i + j] * a[j];
                volatile float p1 = M[12 * k + 4 * i + j] * a[3 + j];
                float mn = std::min((float)p0, (float)p1);
                if (j == 0) s = mn; else s = s + mn;
            }
            volatile float lo = s + M[12 * k + 4 * i + 3];
            std::fesetround(FE_UPWARD);
            volatile float S = 0.0f;
            for (int j = 0; j < 3; ++j) {
                volatile float p0 = M[12 * k + 4 * i + j] * a[j];
                volatile float p1 = M[12 * k + 4 * i + j] * a[3 + j];
                float mx = std::max((float)p0, (float)p1);
                if (j == 0) S = mx; else S = S + mx;
            }
            volatile float hi = S + M[12 * k + 4 * i + 3];
            std::fesetround(old);
            float blo = lo, bhi = hi;
            if (obj_r2) {
                const float* row = M + 12 * (size_t)k + 4 * i;
                float c[3];
                for (int j = 0; j < 3; ++j) c[j] = (a[j] + a[3 + j]) * 0.5f;
                std::fesetround(FE_DOWNWARD);
                volatile float cl = row[0] * c[0];
                volatile float t1 = row[1] * c[1], t2 = row[2] * c[2];
                cl = cl + t1;
                cl = cl + t2;
                cl = cl + row[3];
                std::fesetround(FE_UPWARD);
                volatile float ch = row[0] * c[0];
                volatile float u1 = row[1] * c[1], u2 = row[2] * c[2];
                ch = ch + u1;
                ch = ch + u2;
                ch = ch + row[3];
                volatile float q0 = row[0] * row[0], q1 = row[1] * row[1], q2 = row[2] * row[2];
                volatile float nn = q0 + q1;
                nn = nn + q2;
                volatile float norm = std::sqrt((float)nn);
                volatile float r = std::sqrt(obj_r2[k]);
                volatile float R = r * norm;
                volatile float shi = ch + R;
                std::fesetround(FE_DOWNWARD);
                volatile float slo = cl - R;
                std::fesetround(old);
                blo = std::max((float)lo, (float)slo);
                bhi = std::min((float)hi, (float)shi);
            }
            wbox[6 * (size_t)k + i] = blo;
            wbox[6 * (size_t)k + 3 + i] = bhi;
        }
    }
    std::fesetround(old);
    return rc;
}

// ---- float64 scene -------------------------------------------------------------

void* orc_scene_new(void) { return new Scene(); }
void orc_scene_free(void* s) { delete static_cast<Scene*>(s); }

int orc_scene_add_mesh(void* sp, const float* vtx, uint32_t nv, const uint32_t* idx, uint32_t nt) {
    Scene* S = static_cast<Scene*>(sp);
    Mesh m;
    m.v.resize(nv);
    for (uint32_t i = 0; i < nv; ++i) {
        m.v[i] = V3{vtx[3 * i], vtx[3 * i + 1], vtx[3 * i + 2]};
        m.box.grow(m.v[i]);
        m.vmax = std::max(m.vmax, amax(m.v[i]));
    }
    m.idx.assign(idx, idx + 3 * (size_t)nt);
    m.inv_h.resize(3 * (size_t)nt);
    m.ng.resize(nt);
    std::vector<Box> boxes(nt);
    for (uint32_t p = 0; p < nt; ++p) {
        for (int c = 0; c < 3; ++c)
            if (idx[3 * p + c] >= nv) return -1;
        V3 a = m.v[idx[3 * p]], b = m.v[idx[3 * p + 1]], c = m.v[idx[3 * p + 2]];
        V3 n = cross(b - a, c - a);
        double twoA = norm(n);
        if (twoA > 0) {
            // altitude opposite vertex i = 2*area / |opposite edge|
            m.inv_h[3 * p + 0] = norm(c - b) / twoA;
            m.inv_h[3 * p + 1] = norm(a - c) / twoA;
            m.inv_h[3 * p + 2] = norm(b - a) / twoA;
            m.ng[p] = (1.0 / twoA) * n;
        } else {
            m.inv_h[3 * p + 0] = m.inv_h[3 * p + 1] = m.inv_h[3 * p + 2] = 0.0;
            m.ng[p] = V3{0, 0, 0};
        }
        boxes[p].grow(a);
        boxes[p].grow(b);
        boxes[p].grow(c);
    }
    m.bvh.build(boxes);
    S->meshes.push_back(std::move(m));
    return (int)S->meshes.size() - 1;
}

int orc_scene_set_instances(void* sp, const float* M, const uint32_t* mesh_id, const uint32_t* material_id, uint32_t n) {
    Scene* S = static_cast<Scene*>(sp);
    S->inst.clear();
    std::vector<Box> boxes;
    for (uint32_t k = 0; k < n; ++k) {
        Instance I;
        for (int i = 0; i < 12; ++i) I.M[i] = M[12 * k + i];
        if (mesh_id[k] >= S->meshes.size()) return -1;
        I.mesh = mesh_id[k];
        I.material = material_id ? material_id[k] : 0;
        double det;
        if (!invert34(I.M, I.Minv, &det)) return -2;
        const Box& ob = S->meshes[I.mesh].box;
        for (int c = 0; c < 8; ++c) {
            V3 p{(c & 1) ? ob.hi[0] : ob.lo[0], (c & 2) ? ob.hi[1] : ob.lo[1], (c & 4) ? ob.hi[2] : ob.lo[2]};
            I.wbox.grow(xform_point(I.M, p));
        }
        boxes.push_back(I.wbox);
        S->inst.push_back(I);
    }
    S->tlas.build(boxes);
    return 0;
}

int orc_scene_set_shading(void* sp, const uint32_t* mat_type, const float* albedo, const float* ior, uint32_t nmat,
                          const float* light_pos, const float* light_I, uint32_t nl, const float* background,
                          float ambient) {
    Scene* S = static_cast<Scene*>(sp);
    S->mat_type.assign(mat_type, mat_type + nmat);
    S->mat_albedo.resize(nmat);
    S->mat_ior.resize(nmat);
    for (uint32_t i = 0; i < nmat; ++i) {
        S->mat_albedo[i] = V3{albedo[3 * i], albedo[3 * i + 1], albedo[3 * i + 2]};
        S->mat_ior[i] = ior[i];
    }
    S->light_pos.resize(nl);
    S->light_I.resize(nl);
    for (uint32_t l = 0; l < nl; ++l) {
        S->light_pos[l] = V3{light_pos[3 * l], light_pos[3 * l + 1], light_pos[3 * l + 2]};
        S->light_I[l] = V3{light_I[3 * l], light_I[3 * l + 1], light_I[3 * l + 2]};
    }
    S->background = V3{background[0], background[1], background[2]};
    S->ambient = ambient;
    for (uint32_t k = 0; k < S->inst.size(); ++k)
        if (S->inst[k].material >= nmat) return -1;
    return 0;
}

// Ray queries.  rays: n x {o.xyz, tmin, d.xyz, tmax} float32.
// mode 0 = closest hit, 1 = any hit.  brute = test every triangle.
// kappa scales the float32 error bound eta; rel_t is the relative distance
// tolerance.  Outputs (any may be null): inst/prim (0xFFFFFFFF on miss),
// t (+inf on miss), u (weight of v1), v (weight of v2), ambiguous flag,
// tol_t (distance tolerance), tol_b (barycentric tolerance).  For mode 1,
// inst[i] = 0 if occluded else 0xFFFFFFFF and t/u/v are not written.
int orc_trace(void* sp, const float* rays, int64_t n, int mode, int brute, double kappa, double rel_t, int nthreads,
              uint32_t* inst, uint32_t* prim, double* t, double* u, double* v, uint8_t* amb, double* tol_t,
              double* tol_b) {
    const Scene* S = static_cast<const Scene*>(sp);
    parallel_for(n, nthreads, [&](int64_t i) {
        Query Q(*S, kappa, rel_t);
        const float* r = rays + 8 * i;
        V3 o{r[0], r[1], r[2]}, d{r[4], r[5], r[6]};
        if (mode == 0) {
            QueryOut q = Q.closest(o, d, r[3], r[7], brute != 0);
            if (inst) inst[i] = q.inst;
            if (prim) prim[i] = q.prim;
            if (t) t[i] = q.t;
            if (u) u[i] = q.hit ? q.u : 0.0;
            if (v) v[i] = q.hit ? q.v : 0.0;
            if (amb) amb[i] = q.ambiguous;
            if (tol_t) tol_t[i] = q.tol_t;
            if (tol_b) tol_b[i] = q.tol_b;
        } else {
            bool a = false;
            bool occ = Q.any(o, d, r[3], r[7], brute != 0, &a);
            if (inst) inst[i] = occ ? 0u : 0xFFFFFFFFu;
            if (amb) amb[i] = a;
        }
    });
    return 0;
}

// Primary ray of pixel (x, y) (row 0 = top) for camera {eye.xyz, target.xyz,
// up.xyz, vfov_deg}: float64 pinhole model (see orc_render).
int orc_camera_rays(const float* cam, uint32_t w, uint32_t h, const uint32_t* pix, int64_t n, double* dirs) {
    for (int64_t i = 0; i < n; ++i) {
        V3 d = camera_dir(cam, w, h, pix[i] % w, pix[i] / w);
        dirs[3 * i] = d.x;
        dirs[3 * i + 1] = d.y;
        dirs[3 * i + 2] = d.z;
    }
    return 0;
}

// Whitted render of the listed pixels.  Camera: vertical fov, aspect w/h,
// pixel centre (x+0.5, y+0.5), row 0 at the top, F = normalize(target-eye),
// R = normalize(F x up), U = R x F, d = normalize(px R + py U + F).
// rgba: 4 doubles per listed pixel (alpha = 1 if the primary ray hit);
// amb: 1 if any ray of the pixel's ray tree is ambiguous; counts[0] closest-hit
// rays, counts[1] shadow rays (summed over pixels).
int orc_render(void* sp, const float* cam, uint32_t w, uint32_t h, uint32_t max_depth, const uint32_t* pix, int64_t n,
               double kappa, double rel_t, int nthreads, double* rgba, uint8_t* amb, uint64_t* counts) {
    const Scene* S = static_cast<const Scene*>(sp);
    int nt = nthreads <= 0 ? (int)std::max(1u, std::thread::hardware_concurrency()) : nthreads;
    std::vector<uint64_t> cnt(2 * (size_t)std::max<int64_t>(n, 1), 0);
    parallel_for(n, nt, [&](int64_t i) {
        Query Q(*S, kappa, rel_t);
        Shade sh{*S, Q, (int)max_depth, &cnt[2 * i], false};
        uint32_t x = pix[i] % w, y = pix[i] / w;
        V3 eye{cam[0], cam[1], cam[2]};
        V3 d = camera_dir(cam, w, h, x, y);
        bool hit = false;
        V3 L = sh.trace(eye, d, 1, &hit);
        rgba[4 * i] = L.x;
        rgba[4 * i + 1] = L.y;
        rgba[4 * i + 2] = L.z;
        rgba[4 * i + 3] = hit ? 1.0 : 0.0;
        if (amb) amb[i] = sh.amb;
    });
    if (counts) {
        counts[0] = counts[1] = 0;
        for (int64_t i = 0; i < n; ++i) { counts[0] += cnt[2 * i]; counts[1] += cnt[2 * i + 1]; }
    }
    return 0;
}

// Shading steps, exposed for closed-form checks: reflect (returns 1) and
// refract (returns 1, or 0 on total internal reflection; T and R written).
int orc_reflect(const double* d, const double* nf, double* r) {
    V3 o = reflect_dir(V3{d[0], d[1], d[2]}, V3{nf[0], nf[1], nf[2]});
    r[0] = o.x; r[1] = o.y; r[2] = o.z;
    return 1;
}
int orc_refract(const double* d, const double* nf, int entering, double ior, double* T, double* R) {
    V3 t;
    if (!refract_dir(V3{d[0], d[1], d[2]}, V3{nf[0], nf[1], nf[2]}, entering != 0, ior, &t, R)) return 0;
    T[0] = t.x; T[1] = t.y; T[2] = t.z;
    return 1;
}

// ---------------------------------------------------------------- FXAA
// Fast approximate anti-aliasing (Lottes 2009), float32, one pixel at a time,
// clamp-to-edge addressing, pixel centres at integer coordinates:
//  1. luma = sqrt(max(0.299 R + 0.587 G + 0.114 B, 0)) (a gamma-2 luma of the
//     linear colour);
//  2. skip the pixel (copy it) if the luma range of it and its 4 neighbours
//     is below max(0.0312, 0.125 * the largest of them);
//  3. edge orientation from second differences across the 3x3 block: the
//     edge is horizontal if the vertical differences (weights 1,2,1) are at
//     least the horizontal ones;
//  4. the edge lies toward the neighbour (across the edge) with the larger
//     luma step; the edge luma is the mean of that neighbour and the pixel;
//  5. from half a pixel across (on the edge), step along it both ways (12
//     steps of 1,1,1,1,1,1.5,2,2,2,2,4,8 pixels) until the bilinear luma
//     differs from the edge luma by at least a quarter of the larger step;
//  6. a pixel on the side whose luma change is opposite to the luma found at
//     the nearer edge end moves by 0.5 - (distance to that end) / (edge
//     length) across the edge; every pixel also gets the sub-pixel offset
//     0.75 s^2 with s = smoothstep(|mean of the 3x3 (weights 2 on the 4
//     neighbours, 1 on the corners) - luma| / range);
//  7. the output colour is the bilinear sample at the larger of the two
//     offsets, across the edge; alpha is kept.
namespace fxaa {

struct Img {
    const float* p;
    int w, h;
    int cx(int x) const { return x < 0 ? 0 : (x >= w ? w - 1 : x); }
    int cy(int y) const { return y < 0 ? 0 : (y >= h ? h - 1 : y); }
    float ch(int x, int y, int c) const { return p[4 * ((size_t)cy(y) * (size_t)w + (size_t)cx(x)) + c]; }
    float luma(int x, int y) const {
        const float v = 0.299f * ch(x, y, 0) + 0.587f * ch(x, y, 1) + 0.114f * ch(x, y, 2);
        return std::sqrt(v > 0.0f ? v : 0.0f);
    }
    // bilinear in luma (c < 0) or in channel c, at real pixel coordinates
    float sample(float px, float py, int c) const {
        const float fx0 = std::floor(px), fy0 = std::floor(py);
        const float fx = px - fx0, fy = py - fy0;
        const int x0 = (int)fx0, y0 = (int)fy0;
        auto at = [&](int x, int y) { return c < 0 ? luma(x, y) : ch(x, y, c); };
        const float a = at(x0, y0), b = at(x0 + 1, y0), d = at(x0, y0 + 1), e = at(x0 + 1, y0 + 1);
        const float top = a + fx * (b - a);
        const float bot = d + fx * (e - d);
        return top + fy * (bot - top);
    }
};

const float kEdgeMin = 0.0312f, kEdgeRel = 0.125f, kSubpix = 0.75f;
const float kSteps[12] = {1.0f, 1.0f, 1.0f, 1.0f, 1.0f, 1.5f, 2.0f, 2.0f, 2.0f, 2.0f, 4.0f, 8.0f};

float d2(float a, float m, float b) { return std::fabs((a + b) - 2.0f * m); }

void pixel(const Img& I, int x, int y, float* out) {
    for (int c = 0; c < 4; ++c) out[c] = I.ch(x, y, c);
    const float lM = I.luma(x, y), lN = I.luma(x, y - 1), lS = I.luma(x, y + 1);
    const float lW = I.luma(x - 1, y), lE = I.luma(x + 1, y);
    const float lo = std::min(lM, std::min(std::min(lN, lS), std::min(lW, lE)));
    const float hi = std::max(lM, std::max(std::max(lN, lS), std::max(lW, lE)));
    const float range = hi - lo;
    if (range < std::max(kEdgeMin, hi * kEdgeRel)) return;
    const float lNW = I.luma(x - 1, y - 1), lNE = I.luma(x + 1, y - 1);
    const float lSW = I.luma(x - 1, y + 1), lSE = I.luma(x + 1, y + 1);
    // 3. orientation
    const float eH = (d2(lNW, lW, lSW) + 2.0f * d2(lN, lM, lS)) + d2(lNE, lE, lSE);
    const float eV = (d2(lNW, lN, lNE) + 2.0f * d2(lW, lM, lE)) + d2(lSW, lS, lSE);
    const bool horiz = eH >= eV;
    // 4. side of the edge
    const float l1 = horiz ? lN : lW, l2 = horiz ? lS : lE;
    const float g1 = l1 - lM, g2 = l2 - lM;
    const bool neg = std::fabs(g1) >= std::fabs(g2);
    const float gs = 0.25f * std::max(std::fabs(g1), std::fabs(g2));
    const float lLocal = neg ? 0.5f * (l1 + lM) : 0.5f * (l2 + lM);
    const float sgn = neg ? -1.0f : 1.0f;
    // 5. search along the edge, half a pixel across
    const float fx = (float)x, fy = (float)y;
    const float sx = horiz ? fx : fx + 0.5f * sgn, sy = horiz ? fy + 0.5f * sgn : fy;
    float dist[2] = {0.0f, 0.0f}, end[2] = {0.0f, 0.0f};
    for (int side = 0; side < 2; ++side) {
        const float dir = side == 0 ? -1.0f : 1.0f;
        for (int k = 0; k < 12; ++k) {
            dist[side] = dist[side] + kSteps[k];
            const float px = horiz ? sx + dir * dist[side] : sx;
            const float py = horiz ? sy : sy + dir * dist[side];
            end[side] = I.sample(px, py, -1) - lLocal;
            if (std::fabs(end[side]) >= gs) break;
        }
    }
    // 6. offsets
    const float len = dist[0] + dist[1];
    const bool near0 = dist[0] < dist[1];
    const float dmin = near0 ? dist[0] : dist[1];
    const float eNear = near0 ? end[0] : end[1];
    const float off = ((lM < lLocal) != (eNear < 0.0f)) ? 0.5f - dmin / len : 0.0f;
    const float sum4 = (lN + lS) + (lW + lE);
    const float sumC = (lNW + lNE) + (lSW + lSE);
    const float avg = (2.0f * sum4 + sumC) / 12.0f;
    float sp = std::fabs(avg - lM) / range;
    if (sp > 1.0f) sp = 1.0f;
    sp = ((3.0f - 2.0f * sp) * sp) * sp;
    const float sub = (sp * sp) * kSubpix;
    const float f = std::max(off, sub);
    // 7. resample across the edge
    const float ox = horiz ? fx : fx + f * sgn, oy = horiz ? fy + f * sgn : fy;
    for (int c = 0; c < 3; ++c) out[c] = I.sample(ox, oy, c);
}

}  // namespace fxaa

// FXAA of a w x h RGBA32F image (row 0 at the top) into out (same layout).
int orc_fxaa(const float* rgba, int w, int h, float* out, int threads) {
    if (w <= 0 || h <= 0) return 0;
    const fxaa::Img I{rgba, w, h};
    parallel_for((int64_t)w * h, threads, [&](int64_t i) {
        fxaa::pixel(I, (int)(i % w), (int)(i / w), out + 4 * i);
    });
    return 0;
}

}  // extern "C"
