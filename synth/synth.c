/*
 * Seeded synthetic depth sequences for incremental volumetric meshing.
 *
 * This module generates the INPUTS shared by the CPU oracle and the CUDA path:
 * analytic scenes (spheres, yawed boxes, vertical cylinders, rooms), camera
 * trajectories and noisy float32 depth frames ray-cast with a pinhole camera.
 * It holds none of the meshing method's arithmetic.  It stands in for the
 * RGB-D sequences the paper evaluates on (ICL-NUIM, TUM, Zhou-Koltun; Sec. VI),
 * which are not available: only their shape is mimicked (640x480 float depth,
 * Kinect-like intrinsics, handheld trajectories, depth-dependent noise).
 *
 * Conventions
 *   - World frame is z-up.  Camera frame is OpenCV: x right, y down, z forward.
 *   - Pose T_wc (camera -> world) is a row-major 4x4 double matrix [R | t].
 *   - Depth is camera-z in metres; 0 marks an invalid pixel.
 *   - Pixel (u, v) has its centre at integer coordinates; the ray through it
 *     has camera direction ((u - cx)/fx, (v - cy)/fy, 1).
 *   - Randomness is splitmix64 (Steele, Lea, Flood 2014) with Box-Muller
 *     normals; per-pixel noise is counter based so frames render in any order
 *     and any thread count with identical bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define PI 3.14159265358979323846

enum { P_SPHERE = 0, P_BOX = 1, P_CYL = 2, P_ROOM = 3 };

typedef struct {
  int kind;
  double c[3];  /* centre */
  double h[3];  /* box/room half extents; sphere: h[0]=r; cylinder: h[0]=r, h[2]=half height */
  double yaw, cs, sn;
  double brad; /* bounding-sphere radius (culling) */
} prim_t;

typedef struct {
  int W, H;
  double fx, fy, cx, cy;
  uint64_t seed;
  int nprims, cap;
  prim_t* prims;
  int nframes;
  double* poses; /* nframes x 16, T_wc row-major */
  double noise_const, noise_quad; /* sigma = noise_const + noise_quad * z^2 */
  double invalid_frac;
  double max_range; /* depth beyond it -> 0; <= 0 disables */
  double lo[3], hi[3]; /* scene bounds */
} scene_t;

/* ---------------------------------------------------------------- RNG */
static uint64_t sm64_next(uint64_t* s) {
  uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static double u01(uint64_t* s) { return (double)(sm64_next(s) >> 11) * (1.0 / 9007199254740992.0); }
static double unif(uint64_t* s, double a, double b) { return a + (b - a) * u01(s); }
static double gauss(uint64_t* s) {
  double u1 = u01(s), u2 = u01(s);
  if (u1 < 1e-300) u1 = 1e-300;
  return sqrt(-2.0 * log(u1)) * cos(2.0 * PI * u2);
}

/* ---------------------------------------------------------------- small vector helpers */
static void v_sub(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double v_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void v_cross(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1];
  o[1] = a[2] * b[0] - a[0] * b[2];
  o[2] = a[0] * b[1] - a[1] * b[0];
}
static void v_norm(double* a) {
  double n = sqrt(v_dot(a, a));
  if (n > 0) { a[0] /= n; a[1] /= n; a[2] /= n; }
}

/* ---------------------------------------------------------------- scene building */
static scene_t* scene_new(int W, int H, double fx, double fy, double cx, double cy, uint64_t seed, int nframes) {
  scene_t* s = (scene_t*)calloc(1, sizeof(scene_t));
  s->W = W; s->H = H; s->fx = fx; s->fy = fy; s->cx = cx; s->cy = cy;
  s->seed = seed;
  s->nframes = nframes;
  s->poses = (double*)calloc((size_t)nframes * 16, sizeof(double));
  s->cap = 16;
  s->prims = (prim_t*)calloc(s->cap, sizeof(prim_t));
  return s;
}

static void add_prim(scene_t* s, int kind, double cx, double cy, double cz, double h0, double h1, double h2, double yaw) {
  if (s->nprims == s->cap) {
    s->cap *= 2;
    s->prims = (prim_t*)realloc(s->prims, s->cap * sizeof(prim_t));
  }
  prim_t* p = &s->prims[s->nprims++];
  memset(p, 0, sizeof(*p));
  p->kind = kind;
  p->c[0] = cx; p->c[1] = cy; p->c[2] = cz;
  p->h[0] = h0; p->h[1] = h1; p->h[2] = h2;
  p->yaw = yaw; p->cs = cos(yaw); p->sn = sin(yaw);
  if (kind == P_SPHERE) p->brad = h0;
  else if (kind == P_CYL) p->brad = sqrt(h0 * h0 + h2 * h2);
  else p->brad = sqrt(h0 * h0 + h1 * h1 + h2 * h2);
}

/* Pose looking from `pos` along `fwd` with world z up (OpenCV camera axes). */
static void look_along(const double* pos, const double* fwd_in, double* T) {
  double z[3] = {fwd_in[0], fwd_in[1], fwd_in[2]};
  v_norm(z);
  double up[3] = {0, 0, 1}, x[3], y[3];
  v_cross(z, up, x);
  if (v_dot(x, x) < 1e-12) { double alt[3] = {0, 1, 0}; v_cross(z, alt, x); }
  v_norm(x);
  v_cross(z, x, y);
  for (int r = 0; r < 3; ++r) {
    T[r * 4 + 0] = x[r];
    T[r * 4 + 1] = y[r];
    T[r * 4 + 2] = z[r];
    T[r * 4 + 3] = pos[r];
  }
  T[12] = T[13] = T[14] = 0; T[15] = 1;
}

/* ---------------------------------------------------------------- signed distances */
static void to_local(const prim_t* p, const double* q, double* l) {
  double d[3];
  v_sub(q, p->c, d);
  l[0] = p->cs * d[0] + p->sn * d[1];
  l[1] = -p->sn * d[0] + p->cs * d[1];
  l[2] = d[2];
}

static double box_sdf_local(const double* l, const double* h) {
  double q[3], out = 0, m = -1e300;
  for (int i = 0; i < 3; ++i) {
    q[i] = fabs(l[i]) - h[i];
    double qp = q[i] > 0 ? q[i] : 0;
    out += qp * qp;
    if (q[i] > m) m = q[i];
  }
  return sqrt(out) + (m < 0 ? m : 0);
}

static double prim_sdf(const prim_t* p, const double* q) {
  double l[3];
  switch (p->kind) {
    case P_SPHERE: {
      double d[3];
      v_sub(q, p->c, d);
      return sqrt(v_dot(d, d)) - p->h[0];
    }
    case P_BOX: to_local(p, q, l); return box_sdf_local(l, p->h);
    case P_ROOM: to_local(p, q, l); return -box_sdf_local(l, p->h);
    case P_CYL: {
      double dx = q[0] - p->c[0], dy = q[1] - p->c[1];
      double a = sqrt(dx * dx + dy * dy) - p->h[0];
      double b = fabs(q[2] - p->c[2]) - p->h[2];
      double ap = a > 0 ? a : 0, bp = b > 0 ? b : 0;
      double in = a > b ? a : b;
      return sqrt(ap * ap + bp * bp) + (in < 0 ? in : 0);
    }
  }
  return 1e300;
}

static double scene_sdf(const scene_t* s, const double* q) {
  double best = 1e300;
  for (int i = 0; i < s->nprims; ++i) {
    double d = prim_sdf(&s->prims[i], q);
    if (d < best) best = d;
  }
  return best;
}

/* ---------------------------------------------------------------- ray intersection */
/* Smallest ray parameter t > tmin with o + t d on the primitive's surface, or +inf. */
static double slab(const double* o, const double* d, const double* h, double* tnear, double* tfar) {
  double t0 = -1e300, t1 = 1e300;
  for (int i = 0; i < 3; ++i) {
    if (fabs(d[i]) < 1e-300) {
      if (o[i] < -h[i] || o[i] > h[i]) return 0;
      continue;
    }
    double a = (-h[i] - o[i]) / d[i], b = (h[i] - o[i]) / d[i];
    if (a > b) { double t = a; a = b; b = t; }
    if (a > t0) t0 = a;
    if (b < t1) t1 = b;
  }
  *tnear = t0; *tfar = t1;
  return t0 <= t1;
}

static double prim_hit(const prim_t* p, const double* o, const double* d, double tmin) {
  const double inf = 1e300;
  switch (p->kind) {
    case P_SPHERE: {
      double oc[3];
      v_sub(o, p->c, oc);
      double a = v_dot(d, d), b = 2 * v_dot(d, oc), c = v_dot(oc, oc) - p->h[0] * p->h[0];
      double disc = b * b - 4 * a * c;
      if (disc < 0) return inf;
      double sq = sqrt(disc);
      double t = (-b - sq) / (2 * a);
      if (t > tmin) return t;
      t = (-b + sq) / (2 * a);
      return t > tmin ? t : inf;
    }
    case P_BOX:
    case P_ROOM: {
      double lo[3], ld[3], tn, tf;
      to_local(p, o, lo);
      ld[0] = p->cs * d[0] + p->sn * d[1];
      ld[1] = -p->sn * d[0] + p->cs * d[1];
      ld[2] = d[2];
      if (!slab(lo, ld, p->h, &tn, &tf)) return inf;
      if (p->kind == P_BOX) {
        if (tn > tmin) return tn;
        return inf; /* origin inside a solid box: no visible surface */
      }
      return tf > tmin ? tf : inf;
    }
    case P_CYL: {
      double best = inf;
      double ox = o[0] - p->c[0], oy = o[1] - p->c[1], oz = o[2] - p->c[2];
      double a = d[0] * d[0] + d[1] * d[1];
      if (a > 1e-300) {
        double b = 2 * (ox * d[0] + oy * d[1]), c = ox * ox + oy * oy - p->h[0] * p->h[0];
        double disc = b * b - 4 * a * c;
        if (disc >= 0) {
          double sq = sqrt(disc);
          double ts[2] = {(-b - sq) / (2 * a), (-b + sq) / (2 * a)};
          for (int k = 0; k < 2; ++k) {
            double z = oz + ts[k] * d[2];
            if (ts[k] > tmin && fabs(z) <= p->h[2] && ts[k] < best) best = ts[k];
          }
        }
      }
      if (fabs(d[2]) > 1e-300) {
        for (int sgn = -1; sgn <= 1; sgn += 2) {
          double t = (sgn * p->h[2] - oz) / d[2];
          double x = ox + t * d[0], y = oy + t * d[1];
          if (t > tmin && x * x + y * y <= p->h[0] * p->h[0] && t < best) best = t;
        }
      }
      return best;
    }
  }
  return inf;
}

/* ---------------------------------------------------------------- rendering */
typedef struct { int idx; double near; } cull_t;
static int cmp_cull(const void* a, const void* b) {
  double x = ((const cull_t*)a)->near, y = ((const cull_t*)b)->near;
  return (x > y) - (x < y);
}

static uint64_t pixel_stream(uint64_t seed, int frame, int pix) {
  uint64_t s = seed * 0x2545F4914F6CDD1Dull ^ ((uint64_t)(uint32_t)frame << 32) ^ (uint64_t)(uint32_t)pix;
  sm64_next(&s);
  return s;
}

int synth_render(const scene_t* s, int frame, float* depth) {
  if (frame < 0 || frame >= s->nframes) return -1;
  const double* T = s->poses + (size_t)frame * 16;
  const double o[3] = {T[3], T[7], T[11]};
  /* Cull primitives behind the camera; sort the rest by nearest possible distance. */
  cull_t* order = (cull_t*)malloc(sizeof(cull_t) * (s->nprims > 0 ? s->nprims : 1));
  int n = 0;
  const double fwd[3] = {T[2], T[6], T[10]};
  for (int i = 0; i < s->nprims; ++i) {
    const prim_t* p = &s->prims[i];
    double oc[3];
    v_sub(p->c, o, oc);
    double dist = sqrt(v_dot(oc, oc));
    if (p->kind != P_ROOM && v_dot(oc, fwd) < -p->brad) continue;
    order[n].idx = i;
    order[n].near = p->kind == P_ROOM ? 0.0 : dist - p->brad;
    ++n;
  }
  qsort(order, n, sizeof(cull_t), cmp_cull);
  const int W = s->W, H = s->H;
#pragma omp parallel for schedule(static)
  for (int v = 0; v < H; ++v) {
    for (int u = 0; u < W; ++u) {
      double dc[3] = {(u - s->cx) / s->fx, (v - s->cy) / s->fy, 1.0};
      double d[3];
      for (int r = 0; r < 3; ++r) d[r] = T[r * 4 + 0] * dc[0] + T[r * 4 + 1] * dc[1] + T[r * 4 + 2] * dc[2];
      double dl = sqrt(v_dot(d, d));
      double best = 1e300;
      for (int k = 0; k < n; ++k) {
        /* t is camera z; the world distance along the ray is t * dl */
        if (order[k].near > best * dl) break;
        double t = prim_hit(&s->prims[order[k].idx], o, d, 1e-6);
        if (t < best) best = t;
      }
      int pix = v * W + u;
      float out = 0.0f;
      if (best < 1e299) {
        uint64_t st = pixel_stream(s->seed, frame, pix);
        double z = best;
        double sigma = s->noise_const + s->noise_quad * z * z;
        z += sigma * gauss(&st);
        if (s->invalid_frac > 0 && u01(&st) < s->invalid_frac) z = 0;
        if (s->max_range > 0 && z > s->max_range) z = 0;
        out = z > 0 ? (float)z : 0.0f;
      }
      depth[pix] = out;
    }
  }
  free(order);
  return 0;
}

/* ---------------------------------------------------------------- scene recipes */

/* Sphere r = 0.3 m centred (0, 0, 0.3) on a 2 x 2 m ground square (top face z = 0),
 * camera on a circular orbit of radius 1.2 m about the sphere centre, elevation 30 deg,
 * azimuth theta_k = theta_0 + 2 pi k / 10 + U(-0.05, 0.05), sigma = 1 mm. */
scene_t* synth_create_sphere(uint64_t seed, int nframes, int W, int H, double fx, double fy, double cx, double cy,
                             double noise_sigma) {
  scene_t* s = scene_new(W, H, fx, fy, cx, cy, seed, nframes);
  add_prim(s, P_SPHERE, 0, 0, 0.3, 0.3, 0, 0, 0);
  add_prim(s, P_BOX, 0, 0, -0.05, 1.0, 1.0, 0.05, 0);
  s->noise_const = noise_sigma;
  s->lo[0] = -1; s->lo[1] = -1; s->lo[2] = -0.1;
  s->hi[0] = 1; s->hi[1] = 1; s->hi[2] = 0.6;
  uint64_t st = seed;
  double th0 = unif(&st, 0, 2 * PI);
  const double el = 30.0 * PI / 180.0, R = 1.2;
  const double ctr[3] = {0, 0, 0.3};
  for (int k = 0; k < nframes; ++k) {
    double th = th0 + 2 * PI * k / 10.0 + unif(&st, -0.05, 0.05);
    double pos[3] = {ctr[0] + R * cos(el) * cos(th), ctr[1] + R * cos(el) * sin(th), ctr[2] + R * sin(el)};
    double f[3];
    v_sub(ctr, pos, f);
    look_along(pos, f, s->poses + (size_t)k * 16);
  }
  return s;
}

/* Place `count` random primitives inside [lo, hi] (xy) keeping them `clear` metres away
 * from every point of `keep` (camera positions), sizes U(smin, smax). */
static void place_prims(scene_t* s, uint64_t* st, int count, const double* lo, const double* hi, double zmax,
                        double smin, double smax, const double* keep, int nkeep, double clear) {
  int placed = 0, tries = 0;
  while (placed < count && tries < 200000) {
    ++tries;
    int kind = (int)(u01(st) * 3.0);
    if (kind > 2) kind = 2;
    double a = unif(st, smin, smax) * 0.5, b = unif(st, smin, smax) * 0.5, c = unif(st, smin, smax) * 0.5;
    double yaw = unif(st, 0, 2 * PI);
    double halfz = kind == P_SPHERE ? a : c;
    double m = (kind == P_BOX ? sqrt(a * a + b * b) : a) + 0.02;
    double x = unif(st, lo[0] + m, hi[0] - m), y = unif(st, lo[1] + m, hi[1] - m);
    double z = u01(st) < 0.5 ? lo[2] + halfz : unif(st, lo[2] + 0.5, zmax - halfz - 0.2);
    prim_t tmp;
    memset(&tmp, 0, sizeof(tmp));
    tmp.kind = kind == 0 ? P_SPHERE : (kind == 1 ? P_BOX : P_CYL);
    tmp.c[0] = x; tmp.c[1] = y; tmp.c[2] = z;
    tmp.h[0] = a; tmp.h[1] = kind == 1 ? b : 0; tmp.h[2] = kind == 0 ? 0 : c;
    if (tmp.kind == P_CYL) tmp.h[1] = 0;
    tmp.yaw = yaw; tmp.cs = cos(yaw); tmp.sn = sin(yaw);
    int ok = 1;
    for (int k = 0; k < nkeep && ok; ++k)
      if (prim_sdf(&tmp, keep + 3 * k) < clear) ok = 0;
    if (!ok) continue;
    add_prim(s, tmp.kind, x, y, z, tmp.h[0], tmp.h[1], tmp.h[2], yaw);
    ++placed;
  }
}

/* A room (inverted box) of size sx x sy x sz with `nprims` random boxes/spheres/cylinders
 * (size 0.2-0.8 m, on the floor or floating, random yaw) and a smooth random-walk
 * trajectory: step 1-2 cm/frame with low-pass heading, >= 0.5 m from the walls,
 * height 1.2-1.8 m, view yaw/pitch random-walking. */
scene_t* synth_create_room(uint64_t seed, int nframes, int W, int H, double fx, double fy, double cx, double cy,
                           double sx, double sy, double sz, int nprims, double noise_quad, double invalid_frac) {
  scene_t* s = scene_new(W, H, fx, fy, cx, cy, seed, nframes);
  double lo[3] = {-sx / 2, -sy / 2, 0}, hi[3] = {sx / 2, sy / 2, sz};
  memcpy(s->lo, lo, sizeof(lo));
  memcpy(s->hi, hi, sizeof(hi));
  add_prim(s, P_ROOM, 0, 0, sz / 2, sx / 2, sy / 2, sz / 2, 0);
  s->noise_quad = noise_quad;
  s->invalid_frac = invalid_frac;
  uint64_t st = seed ^ 0xA5A5A5A5ull;
  double margin = 0.5;
  double zlo = 1.2, zhi = sz - 0.3 < 1.8 ? sz - 0.3 : 1.8;
  if (zhi < zlo) zhi = zlo;
  double p[3] = {unif(&st, lo[0] + margin, hi[0] - margin), unif(&st, lo[1] + margin, hi[1] - margin),
                 unif(&st, zlo, zhi)};
  double head = unif(&st, 0, 2 * PI), hrate = 0;
  double yaw = unif(&st, 0, 2 * PI), yrate = 0, pitch = -0.3, prate = 0;
  double* keep = (double*)malloc(sizeof(double) * 3 * (size_t)(nframes > 0 ? nframes : 1));
  for (int k = 0; k < nframes; ++k) {
    hrate = 0.9 * hrate + 0.1 * 0.15 * gauss(&st);
    head += hrate;
    double step = unif(&st, 0.01, 0.02);
    double np[3] = {p[0] + step * cos(head), p[1] + step * sin(head), p[2] + 0.3 * step * gauss(&st)};
    for (int i = 0; i < 2; ++i) {
      double a = lo[i] + margin, b = hi[i] - margin;
      if (np[i] < a || np[i] > b) {
        head = i == 0 ? PI - head : -head;
        np[i] = np[i] < a ? a : b;
      }
    }
    if (np[2] < zlo) np[2] = zlo;
    if (np[2] > zhi) np[2] = zhi;
    memcpy(p, np, sizeof(p));
    yrate = 0.95 * yrate + 0.05 * 0.06 * gauss(&st);
    yaw += yrate;
    prate = 0.95 * prate + 0.05 * 0.03 * gauss(&st);
    pitch += prate;
    if (pitch < -0.6) { pitch = -0.6; prate = 0; }
    if (pitch > 0.1) { pitch = 0.1; prate = 0; }
    double f[3] = {cos(pitch) * cos(yaw), cos(pitch) * sin(yaw), sin(pitch)};
    look_along(p, f, s->poses + (size_t)k * 16);
    memcpy(keep + 3 * k, p, sizeof(p));
  }
  /* keep every 4th camera position clear of primitives by 0.35 m */
  int nk = 0;
  for (int k = 0; k < nframes; k += 4) { memmove(keep + 3 * nk, keep + 3 * k, 3 * sizeof(double)); ++nk; }
  place_prims(s, &st, nprims, lo, hi, sz, 0.2, 0.8, keep, nk, 0.35);
  free(keep);
  return s;
}

/* A 20 x 20 x 4 m floor of 4 x 4 rooms (5 m each) separated by 0.1 m walls with 1 m wide,
 * 2.2 m high doorways in the middle of every wall segment; `per_room` furniture primitives
 * per room; the camera walks a serpentine path through the room centres (and so through
 * the doorways), looking around with a random-walking yaw. */
scene_t* synth_create_floor(uint64_t seed, int nframes, int W, int H, double fx, double fy, double cx, double cy,
                            int per_room, double noise_quad, double invalid_frac, double max_range) {
  const double L = 20, Hh = 4, room = 5, wt = 0.05, door = 0.5, lintel = 2.2;
  scene_t* s = scene_new(W, H, fx, fy, cx, cy, seed, nframes);
  s->lo[0] = -L / 2; s->lo[1] = -L / 2; s->lo[2] = 0;
  s->hi[0] = L / 2; s->hi[1] = L / 2; s->hi[2] = Hh;
  s->noise_quad = noise_quad;
  s->invalid_frac = invalid_frac;
  s->max_range = max_range;
  add_prim(s, P_ROOM, 0, 0, Hh / 2, L / 2, L / 2, Hh / 2, 0);
  for (int axis = 0; axis < 2; ++axis) {
    for (int w = 1; w < 4; ++w) {
      double pos = -L / 2 + w * room;
      for (int seg = 0; seg < 4; ++seg) {
        double a = -L / 2 + seg * room, b = a + room, mid = 0.5 * (a + b);
        double spans[2][2] = {{a, mid - door}, {mid + door, b}};
        for (int k = 0; k < 2; ++k) {
          double c = 0.5 * (spans[k][0] + spans[k][1]), hl = 0.5 * (spans[k][1] - spans[k][0]);
          if (axis == 0) add_prim(s, P_BOX, pos, c, Hh / 2, wt, hl, Hh / 2, 0);
          else add_prim(s, P_BOX, c, pos, Hh / 2, hl, wt, Hh / 2, 0);
        }
        double lz = 0.5 * (lintel + Hh), lh = 0.5 * (Hh - lintel);
        if (axis == 0) add_prim(s, P_BOX, pos, mid, lz, wt, door, lh, 0);
        else add_prim(s, P_BOX, mid, pos, lz, door, wt, lh, 0);
      }
    }
  }
  /* serpentine path through the 16 room centres */
  double path[16][2];
  int np = 0;
  for (int j = 0; j < 4; ++j)
    for (int i = 0; i < 4; ++i) {
      int ii = (j % 2 == 0) ? i : 3 - i;
      path[np][0] = -L / 2 + room * (ii + 0.5);
      path[np][1] = -L / 2 + room * (j + 0.5);
      ++np;
    }
  double total = room * (np - 1);
  uint64_t st = seed ^ 0x5A5A5A5Aull;
  double yaw_off = 0, yrate = 0, pitch = -0.25, prate = 0;
  double* keep = (double*)malloc(sizeof(double) * 3 * (size_t)(nframes > 0 ? nframes : 1));
  for (int k = 0; k < nframes; ++k) {
    double sdist = nframes > 1 ? total * k / (nframes - 1) : 0;
    int seg = (int)(sdist / room);
    if (seg > np - 2) seg = np - 2;
    double f = (sdist - seg * room) / room;
    double p[3] = {path[seg][0] + f * (path[seg + 1][0] - path[seg][0]),
                   path[seg][1] + f * (path[seg + 1][1] - path[seg][1]), 1.5 + 0.1 * sin(0.05 * k)};
    double dir = atan2(path[seg + 1][1] - path[seg][1], path[seg + 1][0] - path[seg][0]);
    yrate = 0.95 * yrate + 0.05 * 0.08 * gauss(&st);
    yaw_off += yrate;
    if (yaw_off > 1.0) { yaw_off = 1.0; yrate = 0; }
    if (yaw_off < -1.0) { yaw_off = -1.0; yrate = 0; }
    prate = 0.95 * prate + 0.05 * 0.03 * gauss(&st);
    pitch += prate;
    if (pitch < -0.6) { pitch = -0.6; prate = 0; }
    if (pitch > 0.05) { pitch = 0.05; prate = 0; }
    double fw[3] = {cos(pitch) * cos(dir + yaw_off), cos(pitch) * sin(dir + yaw_off), sin(pitch)};
    look_along(p, fw, s->poses + (size_t)k * 16);
    memcpy(keep + 3 * k, p, sizeof(p));
  }
  /* path samples every 0.25 m kept clear of furniture */
  int nk = 0;
  double* kp = (double*)malloc(sizeof(double) * 3 * 400);
  for (int i = 0; i + 1 < np; ++i)
    for (int t = 0; t < 20; ++t) {
      double f = t / 20.0;
      kp[3 * nk + 0] = path[i][0] + f * (path[i + 1][0] - path[i][0]);
      kp[3 * nk + 1] = path[i][1] + f * (path[i + 1][1] - path[i][1]);
      kp[3 * nk + 2] = 1.5;
      ++nk;
    }
  for (int j = 0; j < 4; ++j)
    for (int i = 0; i < 4; ++i) {
      double rlo[3] = {-L / 2 + room * i + 0.3, -L / 2 + room * j + 0.3, 0};
      double rhi[3] = {rlo[0] + room - 0.6, rlo[1] + room - 0.6, Hh};
      place_prims(s, &st, per_room, rlo, rhi, Hh, 0.2, 0.8, kp, nk, 0.7);
    }
  free(kp);
  free(keep);
  return s;
}

/* ---------------------------------------------------------------- queries */
void synth_destroy(scene_t* s) {
  if (!s) return;
  free(s->prims);
  free(s->poses);
  free(s);
}
int synth_num_frames(const scene_t* s) { return s->nframes; }
int synth_num_prims(const scene_t* s) { return s->nprims; }
void synth_camera(const scene_t* s, int* W, int* H, double* intr) {
  *W = s->W; *H = s->H;
  intr[0] = s->fx; intr[1] = s->fy; intr[2] = s->cx; intr[3] = s->cy;
}
void synth_bounds(const scene_t* s, double* lo, double* hi) {
  memcpy(lo, s->lo, 3 * sizeof(double));
  memcpy(hi, s->hi, 3 * sizeof(double));
}
int synth_pose(const scene_t* s, int frame, double* T) {
  if (frame < 0 || frame >= s->nframes) return -1;
  memcpy(T, s->poses + (size_t)frame * 16, 16 * sizeof(double));
  return 0;
}
/* Exact scene signed distance (union of the primitives: exact outside the solids,
 * sign-correct inside) and its central-difference gradient (h = 1e-6 m). */
void synth_sdf(const scene_t* s, const double* pts, int n, double* sdf, double* grad) {
  for (int i = 0; i < n; ++i) {
    const double* q = pts + 3 * i;
    sdf[i] = scene_sdf(s, q);
    if (grad) {
      const double h = 1e-6;
      for (int a = 0; a < 3; ++a) {
        double qp[3] = {q[0], q[1], q[2]}, qm[3] = {q[0], q[1], q[2]};
        qp[a] += h; qm[a] -= h;
        grad[3 * i + a] = (scene_sdf(s, qp) - scene_sdf(s, qm)) / (2 * h);
      }
    }
  }
}
