/*
 * FP64 CPU oracle for the stereo ray tracer -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the benchmark's CPU-baseline leg may
 * load this library. It shares no code, header, table or helper with the
 * CUDA path; the two only consume the same seeded scene arrays.
 *
 * What it computes (plain definitions, FP64, no blocking or reordering):
 *
 *  - Stereo camera (Sec. 2-3: two projections of the scene from two cameras
 *    placed at the observer's eyes; Sec. 3 "parallel level 1": the left and
 *    right channel are independent). Off-axis stereo: both eyes share one
 *    image window on the convergence plane.
 *  - Reverse ("classical") ray tracing of every pixel (Sec. 3, Table 1):
 *    primary rays from the eye, shadow rays to every light facing the
 *    surface, mirror reflection rays up to a fixed depth, Whitted shading.
 *    Closest hit = smallest t > 0 over all primitives, equal t -> lower id.
 *    Scenes of <= 64 primitives are brute-forced; larger ones use the
 *    oracle's own BVH (Table 1 lists BVH trees as the GPU-friendly structure).
 *  - The linear BVH ("LBVH") definition: FP64 centroids, 10-bit-per-axis
 *    Morton codes, 64-bit keys (morton << 32 | id), and the binary radix
 *    tree over the sorted keys, produced here top-down by splitting every
 *    key range at its highest differing bit (the same tree the parallel
 *    bottom-up construction defines), plus conservative FP32 boxes.
 *  - Near-tie flags: a ray is flagged when a perturbation of relative size
 *    1e-5 of its scale could change one of its discrete decisions (which
 *    primitive is hit first, whether a shadow ray is blocked, whether a
 *    light faces the surface).
 *
 * Parity status: every function is pinned by tests/test_oracle_*.py
 * (closed forms, invariants, brute force vs BVH, hand-worked radix trees);
 * the paper's own images are lost (its figures are placeholders), so no
 * value of the paper itself pins any output.
 *
 * Build: gcc -O2 -ffp-contract=off -fno-fast-math -shared -fPIC -pthread.
 * -ffp-contract=off is required: the Morton quantisation is specified with
 * every operation correctly rounded and no fused multiply-add.
 */
#include <float.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* --- input records (byte layout of the scene arrays) ------------------- */
typedef struct { float c[3]; float r; uint32_t mat; } osphere;
typedef struct { float v0[3], v1[3], v2[3]; uint32_t mat; } otri;
typedef struct { float albedo[3]; float refl; } omat;
typedef struct { float pos[3]; float intensity; } olight;
typedef struct { float eye[3], fwd[3], up[3]; float vfov_deg; } ocam;

/* shading constants (the paper gives no shading model; these are readings) */
#define K_AMBIENT 0.1
static const double BACKGROUND[3] = {0.2, 0.3, 0.5};
#define TIE_REL 1e-5           /* relative scale of a near-tie decision     */
#define MISS_ID 0xFFFFFFFFu
#define BRUTE_MAX 64           /* brute force up to this many primitives    */

/* ray kinds for counters */
enum { K_PRIMARY = 0, K_SHADOW = 1, K_REFLECT = 2 };

/* ----------------------------------------------------------- vectors --- */
typedef struct { double x, y, z; } v3;
static v3 mk(double x, double y, double z) { v3 r = {x, y, z}; return r; }
static v3 vf(const float* f) { return mk(f[0], f[1], f[2]); }
static v3 add(v3 a, v3 b) { return mk(a.x + b.x, a.y + b.y, a.z + b.z); }
static v3 sub(v3 a, v3 b) { return mk(a.x - b.x, a.y - b.y, a.z - b.z); }
static v3 scl(v3 a, double s) { return mk(a.x * s, a.y * s, a.z * s); }
static double dot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 cross(v3 a, v3 b) {
  return mk(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
static double len(v3 a) { return sqrt(dot(a, a)); }
static v3 unit(v3 a) { return scl(a, 1.0 / len(a)); }
static double ninf(v3 a) { return fmax(fabs(a.x), fmax(fabs(a.y), fabs(a.z))); }
static double comp(v3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

/* ------------------------------------------------------------- scene --- */
typedef struct {
  int32_t left, right;          /* >= 0 internal node, < 0 leaf ~index    */
  float lo[3], hi[3];           /* box of this node                        */
} onode;

typedef struct oscene {
  const osphere* sp; uint32_t ns;
  const otri* tr; uint32_t nt;
  const omat* mat; uint32_t nm;
  const olight* li; uint32_t nl;
  uint32_t n;                   /* ns + nt                                 */
  double scale_max;             /* max |coordinate| over all primitives   */
  /* LBVH (built on demand) */
  uint64_t* keys;               /* sorted keys                             */
  uint32_t* order;              /* leaf k -> primitive id                  */
  onode* inner;                 /* n-1 internal nodes (Karras numbering)   */
  float* leaf_lo; float* leaf_hi; /* n leaf boxes (leaf order)             */
  int32_t* parent;              /* internal i -> [i], leaf k -> [n-1+k]    */
} oscene;

static double prim_scale(const oscene* s, uint32_t id) {
  if (id < s->ns) {
    const osphere* q = &s->sp[id];
    return ninf(vf(q->c)) + q->r;
  }
  const otri* t = &s->tr[id - s->ns];
  return fmax(ninf(vf(t->v0)), fmax(ninf(vf(t->v1)), ninf(vf(t->v2))));
}

/* ============================================================ LBVH ====== */
/* Centroid in FP64, every operation correctly rounded (no FMA). */
static v3 centroid(const oscene* s, uint32_t id) {
  if (id < s->ns) return vf(s->sp[id].c);
  const otri* t = &s->tr[id - s->ns];
  v3 a = vf(t->v0), b = vf(t->v1), c = vf(t->v2);
  v3 m = add(add(a, b), c);
  return mk(m.x / 3.0, m.y / 3.0, m.z / 3.0);
}

static uint32_t quantise(double c, double lo, double hi) {
  double ext = hi - lo;
  if (ext == 0.0) return 0;
  double f = floor((c - lo) / ext * 1024.0);
  if (f > 1023.0) f = 1023.0;
  if (f < 0.0) f = 0.0;
  return (uint32_t)f;
}

/* bit k of x -> 3k+2, of y -> 3k+1, of z -> 3k */
uint32_t oracle_morton30(uint32_t qx, uint32_t qy, uint32_t qz) {
  uint32_t m = 0;
  for (int k = 0; k < 10; ++k) {
    m |= ((qx >> k) & 1u) << (3 * k + 2);
    m |= ((qy >> k) & 1u) << (3 * k + 1);
    m |= ((qz >> k) & 1u) << (3 * k);
  }
  return m;
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return x < y ? -1 : (x > y);
}

static int clz64(uint64_t x) {
  if (x == 0) return 64;
  int n = 0;
  while (!(x & (1ull << 63))) { x <<= 1; ++n; }
  return n;
}

/* smallest float >= a + b (exact sum via TwoSum) */
static float add_round_up(double a, double b) {
  double s = a + b, bb = s - a, err = (a - (s - bb)) + (b - bb);
  float f = (float)s;
  if ((double)f < s || ((double)f == s && err > 0.0)) f = nextafterf(f, INFINITY);
  return f;
}
/* largest float <= a - b */
static float sub_round_down(double a, double b) {
  double s = a - b, bb = s - a, err = (a - (s - bb)) + (-b - bb);
  float f = (float)s;
  if ((double)f > s || ((double)f == s && err < 0.0)) f = nextafterf(f, -INFINITY);
  return f;
}

static void prim_box(const oscene* s, uint32_t id, float lo[3], float hi[3]) {
  if (id < s->ns) {
    const osphere* q = &s->sp[id];
    for (int k = 0; k < 3; ++k) {
      lo[k] = sub_round_down(q->c[k], q->r);
      hi[k] = add_round_up(q->c[k], q->r);
    }
    return;
  }
  const otri* t = &s->tr[id - s->ns];
  for (int k = 0; k < 3; ++k) {
    lo[k] = fminf(t->v0[k], fminf(t->v1[k], t->v2[k]));
    hi[k] = fmaxf(t->v0[k], fmaxf(t->v1[k], t->v2[k]));
  }
}

/* Top-down construction of the radix tree over keys[a..b] (a < b).
 * The node covering [a, b] splits after gamma = the last index whose key
 * shares with keys[a] more leading bits than keys[a] and keys[b] share.
 * Numbering: the left child is node gamma, the right child node gamma + 1
 * (a leaf when its range is a single key); the root is node 0. */
static void build_range(oscene* s, int32_t node, uint32_t a, uint32_t b) {
  int dn = clz64(s->keys[a] ^ s->keys[b]);
  uint32_t gamma = a;
  for (uint32_t i = a; i < b; ++i)
    if (clz64(s->keys[a] ^ s->keys[i]) > dn) gamma = i;
  onode* nd = &s->inner[node];
  uint32_t n = s->n;
  if (gamma == a) { nd->left = ~(int32_t)gamma; s->parent[n - 1 + gamma] = node; }
  else { nd->left = (int32_t)gamma; s->parent[gamma] = node; build_range(s, (int32_t)gamma, a, gamma); }
  if (gamma + 1 == b) { nd->right = ~(int32_t)(gamma + 1); s->parent[n - 1 + gamma + 1] = node; }
  else { nd->right = (int32_t)(gamma + 1); s->parent[gamma + 1] = node; build_range(s, (int32_t)(gamma + 1), gamma + 1, b); }
  /* box = union of the children's boxes */
  float clo[2][3], chi[2][3];
  int32_t ch[2] = {nd->left, nd->right};
  for (int c = 0; c < 2; ++c) {
    if (ch[c] < 0) { memcpy(clo[c], &s->leaf_lo[3 * (uint32_t)~ch[c]], 12); memcpy(chi[c], &s->leaf_hi[3 * (uint32_t)~ch[c]], 12); }
    else { memcpy(clo[c], s->inner[ch[c]].lo, 12); memcpy(chi[c], s->inner[ch[c]].hi, 12); }
  }
  for (int k = 0; k < 3; ++k) { nd->lo[k] = fminf(clo[0][k], clo[1][k]); nd->hi[k] = fmaxf(chi[0][k], chi[1][k]); }
}

static int build_lbvh(oscene* s) {
  if (s->keys) return 0;
  uint32_t n = s->n;
  if (n == 0) return -1;
  s->keys = (uint64_t*)malloc(sizeof(uint64_t) * n);
  s->order = (uint32_t*)malloc(sizeof(uint32_t) * n);
  s->inner = (onode*)calloc(n > 1 ? n - 1 : 1, sizeof(onode));
  s->leaf_lo = (float*)malloc(12 * (size_t)n);
  s->leaf_hi = (float*)malloc(12 * (size_t)n);
  s->parent = (int32_t*)malloc(sizeof(int32_t) * (2 * (size_t)n - 1));
  if (!s->keys || !s->order || !s->inner || !s->leaf_lo || !s->leaf_hi || !s->parent) return -3;
  /* scene bounds of the centroids */
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (uint32_t i = 0; i < n; ++i) {
    v3 c = centroid(s, i);
    for (int k = 0; k < 3; ++k) { lo[k] = fmin(lo[k], comp(c, k)); hi[k] = fmax(hi[k], comp(c, k)); }
  }
  for (uint32_t i = 0; i < n; ++i) {
    v3 c = centroid(s, i);
    uint32_t m = oracle_morton30(quantise(c.x, lo[0], hi[0]), quantise(c.y, lo[1], hi[1]),
                                 quantise(c.z, lo[2], hi[2]));
    s->keys[i] = ((uint64_t)m << 32) | i;
  }
  qsort(s->keys, n, sizeof(uint64_t), cmp_u64);
  for (uint32_t k = 0; k < n; ++k) {
    s->order[k] = (uint32_t)(s->keys[k] & 0xFFFFFFFFu);
    prim_box(s, s->order[k], &s->leaf_lo[3 * k], &s->leaf_hi[3 * k]);
  }
  if (n == 1) { s->parent[0] = -1; return 0; }
  s->parent[0] = -1;
  build_range(s, 0, 0, n - 1);
  return 0;
}

/* ====================================================== intersection ===== */
typedef struct { v3 o, d; } ray;

/* Ray-sphere: roots of |o + t d - c|^2 = r^2, nearest root with t > 0. */
static int hit_sphere(const osphere* q, const ray* r, double* t_out) {
  v3 oc = sub(r->o, vf(q->c));
  double a = dot(r->d, r->d), b = dot(oc, r->d), c = dot(oc, oc) - (double)q->r * q->r;
  double disc = b * b - a * c;
  if (disc < 0.0) return 0;
  double sq = sqrt(disc);
  double t = (-b - sq) / a;
  if (t <= 0.0) t = (-b + sq) / a;
  if (t <= 0.0) return 0;
  *t_out = t;
  return 1;
}

/* Moller-Trumbore: o + t d = v0 + u e1 + v e2, hit iff det != 0, u >= 0,
 * v >= 0, u + v <= 1 (edges inclusive) and t > 0. */
static int hit_tri(const otri* tr, const ray* r, double* t_out) {
  v3 v0 = vf(tr->v0), e1 = sub(vf(tr->v1), v0), e2 = sub(vf(tr->v2), v0);
  v3 p = cross(r->d, e2);
  double det = dot(e1, p);
  if (det == 0.0) return 0;
  double inv = 1.0 / det;
  v3 s = sub(r->o, v0);
  double u = dot(s, p) * inv;
  if (u < 0.0 || u > 1.0) return 0;
  v3 q = cross(s, e1);
  double v = dot(r->d, q) * inv;
  if (v < 0.0 || u + v > 1.0) return 0;
  double t = dot(e2, q) * inv;
  if (t <= 0.0) return 0;
  *t_out = t;
  return 1;
}

static int hit_prim(const oscene* s, uint32_t id, const ray* r, double* t) {
  return id < s->ns ? hit_sphere(&s->sp[id], r, t) : hit_tri(&s->tr[id - s->ns], r, t);
}

/* Distance between segment P0 + s (P1 - P0), s in [0,1] and segment
 * Q0 + t (Q1 - Q0), t in [0,1]: minimise the squared distance over the
 * unit square (interior stationary point, else the best edge of the square). */
static double seg_seg_dist(v3 p0, v3 p1, v3 q0, v3 q1) {
  v3 d1 = sub(p1, p0), d2 = sub(q1, q0), r = sub(p0, q0);
  double a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
  double best = INFINITY;
  /* candidate parameter pairs: stationary point + minimisers on the 4 edges */
  double cand[6][2];
  int nc = 0;
  double b = dot(d1, d2), c = dot(d1, r), den = a * e - b * b;
  if (den > 0.0) { cand[nc][0] = (b * f - c * e) / den; cand[nc][1] = (a * f - b * c) / den; ++nc; }
  for (int side = 0; side < 2; ++side) {
    double sfix = side;                /* s fixed at 0 or 1: t = (b s + f)/e */
    double tt = e > 0.0 ? (b * sfix + f) / e : 0.0;
    cand[nc][0] = sfix; cand[nc][1] = fmin(1.0, fmax(0.0, tt)); ++nc;
    double tfix = side;                /* t fixed: s = (b t - c)/a           */
    double ss = a > 0.0 ? (b * tfix - c) / a : 0.0;
    cand[nc][0] = fmin(1.0, fmax(0.0, ss)); cand[nc][1] = tfix; ++nc;
  }
  for (int k = 0; k < nc; ++k) {
    double sp = cand[k][0], tp = cand[k][1];
    if (sp < 0.0 || sp > 1.0 || tp < 0.0 || tp > 1.0) continue;
    v3 dv = sub(add(p0, scl(d1, sp)), add(q0, scl(d2, tp)));
    best = fmin(best, len(dv));
  }
  return best;
}

/* Could a perturbation of the ray or the primitive by delta change what the
 * ray segment (0, tlim] sees of primitive id?
 *  - the segment passes within delta_k of the primitive's boundary: a
 *    triangle edge, or a sphere's silhouette (closest approach of the ray
 *    line to the centre within delta_k of r, at a parameter inside the
 *    segment);
 *  - the primitive is hit within delta_o of the ray origin, or (for a
 *    primitive other than the closest one) within max(1e-5 t, delta_k) of
 *    the end of the segment;
 *  - the origin lies within delta_o of the primitive's surface.
 * delta_k scales with the primitive's coordinates, delta_o with the
 * origin's (the self-intersection offset is 10 delta_o). */
static int near_boundary(const oscene* s, uint32_t id, const ray* r, double tlim, int is_best,
                         double delta_k, double delta_o) {
  double dl = len(r->d);
  v3 p0 = r->o, p1 = add(r->o, scl(r->d, tlim));
  double t;
  if (hit_prim(s, id, r, &t)) {
    if (t * dl < delta_o) return 1;
    if (!is_best && fabs(t - tlim) * dl <= fmax(TIE_REL * tlim * dl, delta_k)) return 1;
  }
  if (id < s->ns) {
    const osphere* q = &s->sp[id];
    v3 c = vf(q->c);
    double tca = dot(sub(c, r->o), r->d) / (dl * dl);
    double dline = len(sub(c, add(r->o, scl(r->d, tca))));
    if (fabs(dline - (double)q->r) < delta_k && tca * dl > -delta_k && (tca - tlim) * dl < delta_k)
      return 1;
    if (fabs(len(sub(p0, c)) - (double)q->r) < delta_o) return 1;
    return 0;
  }
  const otri* tr = &s->tr[id - s->ns];
  v3 v[3] = {vf(tr->v0), vf(tr->v1), vf(tr->v2)};
  for (int k = 0; k < 3; ++k)
    if (seg_seg_dist(p0, p1, v[k], v[(k + 1) % 3]) < delta_k) return 1;
  /* origin on the triangle (within delta_o of its plane, inside it) */
  v3 n = cross(sub(v[1], v[0]), sub(v[2], v[0]));
  double nl = len(n);
  if (nl > 0.0) {
    n = scl(n, 1.0 / nl);
    double h0 = dot(sub(p0, v[0]), n);
    if (fabs(h0) < delta_o) {
      v3 pp = sub(p0, scl(n, h0));
      int inside = 1;
      for (int k = 0; k < 3; ++k) {
        v3 ek = sub(v[(k + 1) % 3], v[k]);
        if (dot(cross(ek, sub(pp, v[k])), n) / len(ek) < -delta_k) inside = 0;
      }
      if (inside) return 1;
    }
  }
  return 0;
}

/* ========================================================= traversal ===== */
typedef struct {
  uint64_t inner_visits, sphere_tests, tri_tests;
} work_ctr;

/* slab test of box [lo,hi] against ray segment [t0, t1]; returns entry t */
static int slab(const float lo[3], const float hi[3], const ray* r, double t0, double t1,
                double pad, double* tentry) {
  double tn = t0, tf = t1;
  for (int k = 0; k < 3; ++k) {
    double o = comp(r->o, k), d = comp(r->d, k);
    double l = (double)lo[k] - pad, h = (double)hi[k] + pad;
    if (d == 0.0) {
      if (o < l || o > h) return 0;
      continue;
    }
    double ta = (l - o) / d, tb = (h - o) / d;
    if (ta > tb) { double x = ta; ta = tb; tb = x; }
    tn = fmax(tn, ta);
    tf = fmin(tf, tb);
  }
  *tentry = tn;
  return tn <= tf;
}

typedef struct { double t; uint32_t id; } hitrec;

static void consider(hitrec* best, double t, uint32_t id) {
  if (t < best->t || (t == best->t && id < best->id)) { best->t = t; best->id = id; }
}

/* closest hit: brute force */
static hitrec closest_brute(const oscene* s, const ray* r) {
  hitrec best = {INFINITY, MISS_ID};
  for (uint32_t i = 0; i < s->n; ++i) {
    double t;
    if (hit_prim(s, i, r, &t)) consider(&best, t, i);
  }
  return best;
}

/* closest hit: LBVH traversal, nearer child first (equal entry: left first) */
static hitrec closest_bvh(const oscene* s, const ray* r, work_ctr* w) {
  hitrec best = {INFINITY, MISS_ID};
  int32_t stack[160];
  int sp = 0;
  int32_t node = s->n == 1 ? ~0 : 0;
  for (;;) {
    if (node < 0) {
      uint32_t id = s->order[(uint32_t)~node];
      double t;
      if (id < s->ns) w->sphere_tests++; else w->tri_tests++;
      if (hit_prim(s, id, r, &t)) consider(&best, t, id);
    } else {
      const onode* nd = &s->inner[node];
      w->inner_visits++;
      int32_t ch[2] = {nd->left, nd->right};
      double te[2];
      int hitc[2];
      for (int c = 0; c < 2; ++c) {
        const float* lo = ch[c] < 0 ? &s->leaf_lo[3 * (uint32_t)~ch[c]] : s->inner[ch[c]].lo;
        const float* hi = ch[c] < 0 ? &s->leaf_hi[3 * (uint32_t)~ch[c]] : s->inner[ch[c]].hi;
        hitc[c] = slab(lo, hi, r, 0.0, best.t, 0.0, &te[c]);
      }
      if (hitc[0] && hitc[1]) {
        int nearc = te[1] < te[0] ? 1 : 0;
        stack[sp++] = ch[1 - nearc];
        node = ch[nearc];
        continue;
      }
      if (hitc[0] || hitc[1]) { node = hitc[0] ? ch[0] : ch[1]; continue; }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  return best;
}

/* any hit with 0 < t < tmax (shadow rays) */
static int occluded_brute(const oscene* s, const ray* r, double tmax) {
  for (uint32_t i = 0; i < s->n; ++i) {
    double t;
    if (hit_prim(s, i, r, &t) && t < tmax) return 1;
  }
  return 0;
}

static int occluded_bvh(const oscene* s, const ray* r, double tmax, work_ctr* w) {
  int32_t stack[160];
  int sp = 0;
  int32_t node = s->n == 1 ? ~0 : 0;
  for (;;) {
    if (node < 0) {
      uint32_t id = s->order[(uint32_t)~node];
      double t;
      if (id < s->ns) w->sphere_tests++; else w->tri_tests++;
      if (hit_prim(s, id, r, &t) && t < tmax) return 1;
    } else {
      const onode* nd = &s->inner[node];
      w->inner_visits++;
      int32_t ch[2] = {nd->left, nd->right};
      double te[2];
      int hitc[2];
      for (int c = 0; c < 2; ++c) {
        const float* lo = ch[c] < 0 ? &s->leaf_lo[3 * (uint32_t)~ch[c]] : s->inner[ch[c]].lo;
        const float* hi = ch[c] < 0 ? &s->leaf_hi[3 * (uint32_t)~ch[c]] : s->inner[ch[c]].hi;
        hitc[c] = slab(lo, hi, r, 0.0, tmax, 0.0, &te[c]);
      }
      if (hitc[0] && hitc[1]) {
        int nearc = te[1] < te[0] ? 1 : 0;
        stack[sp++] = ch[1 - nearc];
        node = ch[nearc];
        continue;
      }
      if (hitc[0] || hitc[1]) { node = hitc[0] ? ch[0] : ch[1]; continue; }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  return 0;
}

/* Near-tie query along the segment (0, tlim]: is any primitive near a
 * decision boundary (see near_boundary)? best_id is the closest hit of a
 * closest-hit ray (MISS_ID for shadow rays and misses). */
static int ray_near_tie(const oscene* s, int use_bvh, const ray* r, double tlim, uint32_t best_id) {
  double ob = ninf(r->o);
  double dl = len(r->d);
  double delta_o = TIE_REL * fmax(1.0, ob);
  if (!use_bvh) {
    for (uint32_t id = 0; id < s->n; ++id) {
      double delta_k = TIE_REL * fmax(1.0, fmax(ob, prim_scale(s, id)));
      if (near_boundary(s, id, r, tlim, id == best_id, delta_k, delta_o)) return 1;
    }
    return 0;
  }
  /* every primitive whose box, padded by the largest delta_k, meets the
   * padded segment */
  double pad = TIE_REL * fmax(1.0, fmax(ob, s->scale_max));
  int32_t stack[160];
  int sp = 0;
  int32_t node = s->n == 1 ? ~0 : 0;
  for (;;) {
    if (node < 0) {
      uint32_t id = s->order[(uint32_t)~node];
      double delta_k = TIE_REL * fmax(1.0, fmax(ob, prim_scale(s, id)));
      if (near_boundary(s, id, r, tlim, id == best_id, delta_k, delta_o)) return 1;
    } else {
      const onode* nd = &s->inner[node];
      int32_t ch[2] = {nd->left, nd->right};
      double te;
      for (int c = 0; c < 2; ++c) {
        const float* lo = ch[c] < 0 ? &s->leaf_lo[3 * (uint32_t)~ch[c]] : s->inner[ch[c]].lo;
        const float* hi = ch[c] < 0 ? &s->leaf_hi[3 * (uint32_t)~ch[c]] : s->inner[ch[c]].hi;
        if (slab(lo, hi, r, -pad / dl, tlim * (1.0 + TIE_REL) + pad / dl, pad, &te)) stack[sp++] = ch[c];
      }
    }
    if (sp == 0) break;
    node = stack[--sp];
  }
  return 0;
}

/* ============================================================ shading ===== */
typedef struct {
  const oscene* s;
  int use_bvh, max_depth;
  uint64_t rays[3];
  work_ctr work[3];
  int flagged;                  /* any ray of this pixel's tree near a tie */
  int primary_flag;
} tracer;

/* ray length used for the near-tie query of a ray that misses everything */
#define MISS_TLIM 1e7

static v3 trace(tracer* tc, ray r, int depth, int kind, uint32_t* id_out, double* t_out) {
  const oscene* s = tc->s;
  tc->rays[kind]++;
  hitrec h = tc->use_bvh ? closest_bvh(s, &r, &tc->work[kind]) : closest_brute(s, &r);
  double tlim = h.id == MISS_ID ? MISS_TLIM : h.t;
  if (ray_near_tie(s, tc->use_bvh, &r, tlim, h.id)) {
    tc->flagged = 1;
    if (kind == K_PRIMARY) tc->primary_flag = 1;
  }
  if (id_out) *id_out = h.id;
  if (t_out) *t_out = h.t;
  if (h.id == MISS_ID) return mk(BACKGROUND[0], BACKGROUND[1], BACKGROUND[2]);

  v3 p = add(r.o, scl(r.d, h.t));
  v3 n;
  uint32_t mid;
  if (h.id < s->ns) {
    const osphere* q = &s->sp[h.id];
    n = scl(sub(p, vf(q->c)), 1.0 / q->r);
    mid = q->mat;
  } else {
    const otri* t = &s->tr[h.id - s->ns];
    v3 v0 = vf(t->v0);
    n = unit(cross(sub(vf(t->v1), v0), sub(vf(t->v2), v0)));
    mid = t->mat;
  }
  if (dot(n, r.d) > 0.0) n = scl(n, -1.0);
  const omat* m = &s->mat[mid];
  v3 alb = vf(m->albedo);
  double eps = 1e-4 * fmax(1.0, ninf(p));
  v3 o2 = add(p, scl(n, eps));

  double lsum = K_AMBIENT;
  for (uint32_t l = 0; l < s->nl; ++l) {
    v3 lv = sub(vf(s->li[l].pos), o2);
    double ld = len(lv);
    v3 lhat = scl(lv, 1.0 / ld);
    double ndl = dot(n, lhat);
    if (fabs(ndl) < TIE_REL) tc->flagged = 1;
    if (ndl <= 0.0) continue;
    tc->rays[K_SHADOW]++;
    ray sr = {o2, lhat};
    double tmax = ld - eps;
    int occ = tc->use_bvh ? occluded_bvh(s, &sr, tmax, &tc->work[K_SHADOW])
                          : occluded_brute(s, &sr, tmax);
    if (ray_near_tie(s, tc->use_bvh, &sr, tmax, MISS_ID)) tc->flagged = 1;
    if (!occ) lsum += (double)s->li[l].intensity * ndl;
  }
  v3 local = scl(alb, lsum);
  double refl = m->refl;
  v3 col = scl(local, 1.0 - refl);
  if (refl > 0.0 && depth < tc->max_depth) {
    v3 rd = unit(sub(r.d, scl(n, 2.0 * dot(r.d, n))));
    ray rr = {o2, rd};
    v3 c2 = trace(tc, rr, depth + 1, K_REFLECT, NULL, NULL);
    col = add(col, scl(c2, refl));
  }
  return col;
}

/* ============================================================= camera ===== */
typedef struct {
  v3 eye, fwd, right, up;
  double tanh_y, aspect, zc, sep;
  int W, H;
} ocamera;

static ocamera setup_camera(const ocam* c, double eye_sep, double convergence, int W, int H) {
  ocamera k;
  k.eye = vf(c->eye);
  k.fwd = unit(vf(c->fwd));
  k.right = unit(cross(vf(c->fwd), vf(c->up)));
  k.up = cross(k.right, k.fwd);
  k.tanh_y = tan(0.5 * (double)c->vfov_deg * M_PI / 180.0);
  k.aspect = (double)W / (double)H;
  k.zc = convergence;
  k.sep = eye_sep;
  k.W = W;
  k.H = H;
  return k;
}

/* Off-axis stereo: both eyes aim at the same point Q of the shared window
 * on the convergence plane. eye = -1 (left) or +1 (right). */
static ray primary_ray(const ocamera* k, int eye, int i, int j) {
  double nx = (2.0 * (i + 0.5) / k->W - 1.0) * k->tanh_y * k->aspect;
  double ny = (1.0 - 2.0 * (j + 0.5) / k->H) * k->tanh_y;
  v3 q = add(k->eye, scl(add(k->fwd, add(scl(k->right, nx), scl(k->up, ny))), k->zc));
  v3 o = add(k->eye, scl(k->right, eye * 0.5 * k->sep));
  ray r = {o, unit(sub(q, o))};
  return r;
}

/* ========================================================== public API ==== */
oscene* oracle_scene_new(const osphere* sp, uint32_t ns, const otri* tr, uint32_t nt,
                         const omat* mat, uint32_t nm, const olight* li, uint32_t nl) {
  oscene* s = (oscene*)calloc(1, sizeof(oscene));
  if (!s) return NULL;
  s->sp = sp; s->ns = ns; s->tr = tr; s->nt = nt; s->mat = mat; s->nm = nm; s->li = li; s->nl = nl;
  s->n = ns + nt;
  s->scale_max = 1.0;
  for (uint32_t i = 0; i < s->n; ++i) s->scale_max = fmax(s->scale_max, prim_scale(s, i));
  return s;
}

void oracle_scene_free(oscene* s) {
  if (!s) return;
  free(s->keys); free(s->order); free(s->inner); free(s->leaf_lo); free(s->leaf_hi); free(s->parent);
  free(s);
}

/* LBVH arrays: keys[n] sorted; left/right[n-1] (child >= 0 internal, < 0
 * leaf ~k); parent[2n-1] (internal i at [i], leaf k at [n-1+k], root -1);
 * inner_box[(n-1)*6] and leaf_box[n*6] as lo xyz, hi xyz. */
int oracle_lbvh(oscene* s, uint64_t* keys, int32_t* left, int32_t* right, int32_t* parent,
                float* inner_box, float* leaf_box) {
  int rc = build_lbvh(s);
  if (rc) return rc;
  uint32_t n = s->n;
  if (keys) memcpy(keys, s->keys, 8 * (size_t)n);
  for (uint32_t i = 0; i + 1 < n; ++i) {
    if (left) left[i] = s->inner[i].left;
    if (right) right[i] = s->inner[i].right;
    if (inner_box) { memcpy(&inner_box[6 * i], s->inner[i].lo, 12); memcpy(&inner_box[6 * i + 3], s->inner[i].hi, 12); }
  }
  if (parent) memcpy(parent, s->parent, 4 * (2 * (size_t)n - 1));
  if (leaf_box)
    for (uint32_t k = 0; k < n; ++k) { memcpy(&leaf_box[6 * k], &s->leaf_lo[3 * k], 12); memcpy(&leaf_box[6 * k + 3], &s->leaf_hi[3 * k], 12); }
  return 0;
}

/* single-ray query (for closed-form pins): closest hit of o + t d */
int oracle_closest(oscene* s, const double o[3], const double d[3], int mode, double* t,
                   uint32_t* id, int* near_tie) {
  int use_bvh = mode == 2 || (mode == 0 && s->n > BRUTE_MAX);
  if (use_bvh && build_lbvh(s)) return -1;
  ray r = {mk(o[0], o[1], o[2]), mk(d[0], d[1], d[2])};
  work_ctr w = {0, 0, 0};
  hitrec h = use_bvh ? closest_bvh(s, &r, &w) : closest_brute(s, &r);
  *t = h.t;
  *id = h.id;
  if (near_tie) *near_tie = ray_near_tie(s, use_bvh, &r, h.id == MISS_ID ? MISS_TLIM : h.t, h.id);
  return 0;
}

typedef struct {
  int W, H, max_depth, mode, n_threads;
  double eye_sep, convergence;
  const int64_t* pixels; int64_t n_pixels;  /* index = eye*W*H + j*W + i; NULL = all */
} oparams;

typedef struct {
  double* rgb;       /* n x 3                                   */
  uint32_t* hit_id;  /* n: primary hit primitive or 0xFFFFFFFF  */
  double* depth;     /* n: view depth of the primary hit, +inf  */
  uint8_t* flags;    /* n: bit0 primary near-tie, bit1 any ray  */
  uint64_t* rays;    /* [3] primary, shadow, reflection         */
  uint64_t* work;    /* [9] per kind: inner visits, sphere, tri */
} oout;

typedef struct {
  oscene* s;
  const ocamera* cam;
  const oparams* p;
  oout* out;
  int use_bvh;
  int64_t next;      /* shared work counter (atomic)            */
  pthread_mutex_t mu;
} job;

static void* worker(void* arg) {
  job* jb = (job*)arg;
  const oparams* p = jb->p;
  int64_t total = p->pixels ? p->n_pixels : 2ll * p->W * p->H;
  uint64_t rays[3] = {0, 0, 0}, work[9] = {0};
  const int64_t chunk = 64;
  for (;;) {
    int64_t b = __atomic_fetch_add(&jb->next, chunk, __ATOMIC_RELAXED);
    if (b >= total) break;
    int64_t e = b + chunk < total ? b + chunk : total;
    for (int64_t k = b; k < e; ++k) {
      int64_t pix = p->pixels ? p->pixels[k] : k;
      int64_t per = (int64_t)p->W * p->H;
      int eye = (int)(pix / per);
      int64_t rem = pix % per;
      int j = (int)(rem / p->W), i = (int)(rem % p->W);
      tracer tc;
      memset(&tc, 0, sizeof tc);
      tc.s = jb->s; tc.use_bvh = jb->use_bvh; tc.max_depth = p->max_depth;
      ray r = primary_ray(jb->cam, eye ? 1 : -1, i, j);
      uint32_t id;
      double t;
      v3 c = trace(&tc, r, 0, K_PRIMARY, &id, &t);
      if (jb->out->rgb) {
        jb->out->rgb[3 * k + 0] = fmin(1.0, fmax(0.0, c.x));
        jb->out->rgb[3 * k + 1] = fmin(1.0, fmax(0.0, c.y));
        jb->out->rgb[3 * k + 2] = fmin(1.0, fmax(0.0, c.z));
      }
      if (jb->out->hit_id) jb->out->hit_id[k] = id;
      if (jb->out->depth) jb->out->depth[k] = id == MISS_ID ? INFINITY : t * dot(r.d, jb->cam->fwd);
      if (jb->out->flags) jb->out->flags[k] = (uint8_t)(tc.primary_flag | (tc.flagged << 1));
      for (int q = 0; q < 3; ++q) {
        rays[q] += tc.rays[q];
        work[3 * q + 0] += tc.work[q].inner_visits;
        work[3 * q + 1] += tc.work[q].sphere_tests;
        work[3 * q + 2] += tc.work[q].tri_tests;
      }
    }
  }
  pthread_mutex_lock(&jb->mu);
  if (jb->out->rays) for (int q = 0; q < 3; ++q) jb->out->rays[q] += rays[q];
  if (jb->out->work) for (int q = 0; q < 9; ++q) jb->out->work[q] += work[q];
  pthread_mutex_unlock(&jb->mu);
  return NULL;
}

int oracle_render(oscene* s, const ocam* c, const oparams* p, oout* out) {
  if (!s || !c || !p || !out || p->W < 1 || p->H < 1 || p->max_depth < 0) return -1;
  int use_bvh = p->mode == 2 || (p->mode == 0 && s->n > BRUTE_MAX);
  if (use_bvh && build_lbvh(s)) return -3;
  ocamera cam = setup_camera(c, p->eye_sep, p->convergence, p->W, p->H);
  if (out->rays) memset(out->rays, 0, 3 * sizeof(uint64_t));
  if (out->work) memset(out->work, 0, 9 * sizeof(uint64_t));
  job jb;
  jb.s = s; jb.cam = &cam; jb.p = p; jb.out = out; jb.use_bvh = use_bvh; jb.next = 0;
  pthread_mutex_init(&jb.mu, NULL);
  int nt = p->n_threads > 0 ? p->n_threads : 1;
  if (nt > 256) nt = 256;
  pthread_t th[256];
  for (int i = 1; i < nt; ++i) pthread_create(&th[i], NULL, worker, &jb);
  worker(&jb);
  for (int i = 1; i < nt; ++i) pthread_join(th[i], NULL);
  pthread_mutex_destroy(&jb.mu);
  return 0;
}

/* primary ray of pixel (i, j) of eye -1 (left) / +1 (right), for pins */
void oracle_primary_ray(const ocam* c, double eye_sep, double convergence, int W, int H, int eye,
                        int i, int j, double o[3], double d[3]) {
  ocamera k = setup_camera(c, eye_sep, convergence, W, H);
  ray r = primary_ray(&k, eye, i, j);
  o[0] = r.o.x; o[1] = r.o.y; o[2] = r.o.z;
  d[0] = r.d.x; d[1] = r.d.y; d[2] = r.d.z;
}
