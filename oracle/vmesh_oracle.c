/*
 * TEST INFRASTRUCTURE ONLY.  Plain, slow, single-threaded CPU oracle of the
 * per-frame hot path of incremental volumetric meshing (Dong, Shi, Tang, Wang,
 * Zha, "An Efficient Volumetric Mesh Representation for Real-time Scene
 * Reconstruction using Spatial Hashing", arXiv 1803.03949).  Only the tests,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the product
 * path never does.  It shares no code with the CUDA library.
 *
 * Compiled twice from this one file:
 *   OR_REAL=float   the parity build: every floating-point decision that fixes
 *                   an integer result (block set, cube codes, refinement) is
 *                   taken in float32 with the operation order written below,
 *                   no contraction (-ffp-contract=off), IEEE division and sqrt;
 *   OR_REAL=double  the error statement: the same steps in float64.
 *
 * What it computes (paper passages and the readings taken where the paper is silent):
 *   - Lattice (Sec. IV): a voxel is a cube corner; global voxel g sits at world
 *     g * l; 8^3 voxels per block; block key b = floor(g / 8); cube g has corners
 *     g + {0,1}^3 in Bourke order 0:(000) 1:(100) 2:(110) 3:(010) 4:(001) 5:(101)
 *     6:(111) 7:(011); cube bit k is corner k.  Voxel g owns the three edges
 *     g -> g + e_x, e_y, e_z (Sec. IV, "1 corner and 3 edges per cube").
 *   - Block collection (Sec. V-A, Eq. 1): for each valid pixel (depth finite and
 *     > 0) the ray segment between camera depths max(D - mu, 0.05) and D + mu is
 *     walked with a 3D DDA over block cells (all cells from the start cell to the
 *     end cell, ties x before y before z); every cell visited is collected and
 *     allocated if new.  Each division is a product with a reciprocal (of fx, fy,
 *     the block side 8 l, and of each axis direction of the segment).
 *   - Fusion (Sec. V-A, Eq. 2, averaging as in Newcombe et al. 2011): every
 *     voxel of the blocks collected by this frame is projected (pinhole,
 *     nearest pixel = floor(u + 0.5)); sdf = D - z_c; skipped when z_c <= 0,
 *     outside the image, invalid depth or sdf < -mu; d~ = min(sdf, mu); w = 1;
 *     d <- (d W + d~) / (W + 1), W <- min(W + 1, W_max).
 *   - Cube type (Sec. V-B): a cube is valid iff all 8 corners are allocated with
 *     W > 0; t = sum_k [d(c_k) < 0] 2^k; an invalid cube has effective type 0.
 *   - Update set: blocks collected since the last mesh update plus their existing
 *     neighbours at offsets {0,-1}^3 \ {0} (their border cubes read corners in
 *     the collected blocks).
 *   - Marching-cubes table T (Sec. V-B): built here from its definition: on each
 *     cube face pair the sign-change edges; on a face with four sign changes the
 *     negative corners are cut off separately; segments are oriented so that the
 *     surface normal points from negative to positive TSDF; each closed loop is
 *     fanned from its smallest edge id whose fan diagonals join no two edges of a
 *     common face (no triangle or diagonal lies in a cube face, so a face segment
 *     is shared by exactly two triangles).  The same face rule on both sides of a
 *     face makes the mesh watertight.
 *   - Vertex (Sec. V-C): on owned edge g -> g + e_a, t = d0 / (d0 - d1) (0.5
 *     when d0 == d1), clamped to [-1, 2] (refined cubes extrapolate, Sec. V-F);
 *     position g*l + t*l*e_a; normal = normalised gradient of the trilinear
 *     interpolant of the owner cube g at the vertex (component b != a uses the
 *     corners g+e_b, g+e_a+e_b; 0 if either is unusable).
 *   - Triangulation (Sec. V-D): a cube's triangles are T(effective type) on
 *     edge-owned vertices; they are kept while the effective type is unchanged.
 *   - Refinement (Sec. V-F, Eqs. 3-5): for a valid cube with raw type t_i and
 *     previous effective type t_{i-1}: if d_H(t_i, t_{i-1}) <= 3, among the six
 *     regular types t_rj with d_H(t_i, t_rj) <= 3 and |d(c_k)| < eps at every
 *     differing corner k, the nearest (ties: lowest j) replaces t_i.
 *   - Garbage collection (Sec. V-E): vertices exist exactly while referenced, so
 *     they need no separate state here.  A block is freed when it was not
 *     collected since the last epoch change, no cube of it or of its 7 lower
 *     neighbours has triangles, none of its voxels owns a referenced edge, and
 *     every voxel has W = 0 or d >= mu.  The paper recycles vertices only; block
 *     recycling is this implementation's addition.  A gc between a frame's
 *     integration and its mesh update keeps the pending update set; a gc after the
 *     mesh update empties the update set (a refinement pass after gc does nothing).
 *   - Differentiable path (the reading taken for gradients through Secs. V-A and V-C,
 *     topology held fixed): between or_diff_begin and the gradient calls every
 *     integration of a voxel is recorded with its frame, pixel, pre-update weight W
 *     and whether d~ = sdf (sdf < mu; d~ = mu is constant in the depth).  Gradients
 *     of a loss given by its derivatives at the vertex positions and normals flow
 *     (or_grad_vertices) into the TSDF values through the edge interpolation and the
 *     normal above, and (or_grad_depth) from the TSDF values to the depth pixels by
 *     reverse-mode through d <- (d W + d~) / (W + 1): per recorded integration,
 *     taken last to first, dL/dd~ = g / (W + 1) reaches the pixel when d~ = sdf, and
 *     g <- g W / (W + 1).  Decisions (which voxel, pixel, branch) are this build's;
 *     the derivative arithmetic is float64 in both builds.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef OR_REAL
#define OR_REAL double
#endif
typedef OR_REAL real;
#define OR_IS_FLOAT (sizeof(real) == sizeof(float))
static real real_sqrt(real x) { return OR_IS_FLOAT ? (real)sqrtf((float)x) : (real)sqrt((double)x); }

#define BS 8
#define BV 512
#define ZMIN ((real)0.05)
#define KEY_LIM ((1 << 20) - 2)

/* ------------------------------------------------------------ cube geometry (Sec. IV) */
static const int CORNER[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
                                 {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
/* edge k joins corner EDGE[k][0] (the owner, lower coordinate) to EDGE[k][1] */
static const int EDGE[12][2] = {{0, 1}, {1, 2}, {3, 2}, {0, 3}, {4, 5}, {5, 6},
                                {7, 6}, {4, 7}, {0, 4}, {1, 5}, {2, 6}, {3, 7}};
/* the 6 faces, corners in cyclic order, with outward normals */
static const int FACE[6][4] = {{0, 3, 7, 4}, {1, 2, 6, 5}, {0, 1, 5, 4}, {3, 2, 6, 7}, {0, 1, 2, 3}, {4, 5, 6, 7}};
static const int FACE_N[6][3] = {{-1, 0, 0}, {1, 0, 0}, {0, -1, 0}, {0, 1, 0}, {0, 0, -1}, {0, 0, 1}};
/* regular cube types of Sec. V-F, read as binary numbers (bit 7 first) */
static const int REGULAR[6] = {0xCC, 0x33, 0x99, 0x66, 0xF0, 0x0F};

static int edge_axis(int k) {
  const int* a = CORNER[EDGE[k][0]];
  const int* b = CORNER[EDGE[k][1]];
  for (int i = 0; i < 3; ++i)
    if (a[i] != b[i]) return i;
  return -1;
}
static int edge_between(int a, int b) {
  for (int k = 0; k < 12; ++k)
    if ((EDGE[k][0] == a && EDGE[k][1] == b) || (EDGE[k][0] == b && EDGE[k][1] == a)) return k;
  return -1;
}

static int edge_on_face(int k, int f) {
  int a = 0, b = 0;
  for (int i = 0; i < 4; ++i) a |= FACE[f][i] == EDGE[k][0], b |= FACE[f][i] == EDGE[k][1];
  return a && b;
}
static int edges_share_face(int j, int k) {
  for (int f = 0; f < 6; ++f)
    if (edge_on_face(j, f) && edge_on_face(k, f)) return 1;
  return 0;
}

static int tri_n[256];
static int tri_e[256][5][3];
static int table_ok = -1;

/* Build the triangle table T from the face rule (see header).  Returns 1 if every
 * sign-change edge received exactly one outgoing and one incoming segment. */
static int build_table(void) {
  int ok = 1;
  for (int code = 0; code < 256; ++code) {
    int next[12], nout[12], nin[12];
    for (int k = 0; k < 12; ++k) next[k] = -1, nout[k] = 0, nin[k] = 0;
    for (int f = 0; f < 6; ++f) {
      const int* q = FACE[f];
      int neg[4];
      for (int i = 0; i < 4; ++i) neg[i] = (code >> q[i]) & 1;
      int segs[2][2], ns = 0, cross[4], nc = 0;
      for (int i = 0; i < 4; ++i)
        if (neg[i] != neg[(i + 1) % 4]) cross[nc++] = edge_between(q[i], q[(i + 1) % 4]);
      if (nc == 2) {
        segs[0][0] = cross[0]; segs[0][1] = cross[1]; ns = 1;
      } else if (nc == 4) {
        for (int i = 0; i < 4; ++i)
          if (neg[i]) {
            segs[ns][0] = edge_between(q[(i + 3) % 4], q[i]);
            segs[ns][1] = edge_between(q[i], q[(i + 1) % 4]);
            ++ns;
          }
      }
      for (int s = 0; s < ns; ++s) {
        int p = segs[s][0], r = segs[s][1];
        /* doubled integer coordinates: edge midpoints and the negative corner of edge p */
        int P[3], Q[3], Wc[3], u[3], w[3], c[3];
        int wn = ((code >> EDGE[p][0]) & 1) ? EDGE[p][0] : EDGE[p][1];
        for (int i = 0; i < 3; ++i) {
          P[i] = CORNER[EDGE[p][0]][i] + CORNER[EDGE[p][1]][i];
          Q[i] = CORNER[EDGE[r][0]][i] + CORNER[EDGE[r][1]][i];
          Wc[i] = 2 * CORNER[wn][i];
          u[i] = Q[i] - P[i];
          w[i] = Wc[i] - P[i];
        }
        c[0] = u[1] * w[2] - u[2] * w[1];
        c[1] = u[2] * w[0] - u[0] * w[2];
        c[2] = u[0] * w[1] - u[1] * w[0];
        int sgn = c[0] * FACE_N[f][0] + c[1] * FACE_N[f][1] + c[2] * FACE_N[f][2];
        if (sgn > 0) { int t = p; p = r; r = t; }
        if (sgn == 0) ok = 0;
        next[p] = r;
        nout[p]++;
        nin[r]++;
      }
    }
    for (int k = 0; k < 12; ++k) {
      int crossing = ((code >> EDGE[k][0]) & 1) != ((code >> EDGE[k][1]) & 1);
      if (crossing ? (nout[k] != 1 || nin[k] != 1) : (nout[k] != 0 || nin[k] != 0)) ok = 0;
    }
    int used[12] = {0}, nt = 0;
    for (int s = 0; s < 12; ++s) {
      if (next[s] < 0 || used[s]) continue;
      int loop[12], len = 0, e = s;
      while (!used[e] && len < 12) { used[e] = 1; loop[len++] = e; e = next[e]; }
      if (e != s) ok = 0;
      /* fan apex: the smallest edge id whose fan diagonals join no two edges of a
       * common face (a diagonal on a face would be shared with the neighbouring cube) */
      int apex = -1;
      for (int a = 0; a < len; ++a) {
        int good = 1;
        for (int i = 2; i + 1 < len; ++i)
          if (edges_share_face(loop[a], loop[(a + i) % len])) good = 0;
        if (good && (apex < 0 || loop[a] < loop[apex])) apex = a;
      }
      if (apex < 0) { ok = 0; apex = 0; }
      for (int i = 1; i + 1 < len; ++i) {
        if (nt >= 5) { ok = 0; break; }
        tri_e[code][nt][0] = loop[apex];
        tri_e[code][nt][1] = loop[(apex + i) % len];
        tri_e[code][nt][2] = loop[(apex + i + 1) % len];
        ++nt;
      }
    }
    tri_n[code] = nt;
  }
  return ok;
}

static void ensure_table(void) {
  if (table_ok < 0) table_ok = build_table();
}

/* ------------------------------------------------------------ blocks and the block map */
typedef struct {
  int key[3];
  int alive;
  unsigned touch_stamp; /* integrate call that last collected it */
  unsigned touch_epoch; /* mesh epoch in which it was last collected */
  int mark;             /* scratch flag for set building */
  real tsdf[BV];
  real weight[BV];
  unsigned char code_eff[BV];
  unsigned char code_prev[BV];
  double gd[BV]; /* dL/dd of the differentiable path */
} oblock;

/* one recorded integration of the differentiable path */
typedef struct {
  int block, voxel, frame, pixel;
  double wpre;       /* weight before the update */
  unsigned char lin; /* d~ = sdf (1) or d~ = mu (0) */
} orec;

typedef struct {
  real l, mu, eps, wmax;
  int64_t* mkeys;
  int* mvals;
  int64_t mcap, mcount;
  oblock** blocks;
  int nblocks, bcap;
  unsigned frame, epoch;
  int advance_pending;
  int *pending, npending, pcap;
  int *last_set, nlast, lcap;
  int *frame_list, nframe, fcap;
  int64_t stat_cells, stat_voxels_integrated, stat_truncated;
  /* differentiable path: recording switch, recorded integrate calls, records */
  int diff_on, diff_frames;
  orec* recs;
  int64_t nrec, rcap;
  /* mesh export scratch */
  uint64_t* vkeys;
  double *vpos, *vnrm;
  uint64_t* tkeys;
  int64_t nv, nt;
} ovol;

static int64_t pack_block(int x, int y, int z) {
  return ((int64_t)(x + (1 << 20)) << 42) | ((int64_t)(y + (1 << 20)) << 21) | (int64_t)(z + (1 << 20));
}
static uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 33)) * 0xFF51AFD7ED558CCDull;
  z = (z ^ (z >> 33)) * 0xC4CEB9FE1A85EC53ull;
  return z ^ (z >> 33);
}
static int floordiv8(int g) { return g >= 0 ? g / 8 : -((-g + 7) / 8); }

static void push_int(int** arr, int* n, int* cap, int v) {
  if (*n == *cap) {
    *cap = *cap ? *cap * 2 : 64;
    *arr = (int*)realloc(*arr, sizeof(int) * (size_t)*cap);
  }
  (*arr)[(*n)++] = v;
}

static void map_rebuild(ovol* V, int64_t cap) {
  free(V->mkeys);
  free(V->mvals);
  V->mcap = cap;
  V->mkeys = (int64_t*)malloc(sizeof(int64_t) * (size_t)cap);
  V->mvals = (int*)malloc(sizeof(int) * (size_t)cap);
  for (int64_t i = 0; i < cap; ++i) V->mkeys[i] = -1;
  V->mcount = 0;
  for (int b = 0; b < V->nblocks; ++b) {
    if (!V->blocks[b]->alive) continue;
    int64_t k = pack_block(V->blocks[b]->key[0], V->blocks[b]->key[1], V->blocks[b]->key[2]);
    int64_t s = (int64_t)(mix64((uint64_t)k) & (uint64_t)(cap - 1));
    while (V->mkeys[s] != -1) s = (s + 1) & (cap - 1);
    V->mkeys[s] = k;
    V->mvals[s] = b;
    V->mcount++;
  }
}

static int find_block(const ovol* V, int x, int y, int z) {
  int64_t k = pack_block(x, y, z);
  int64_t s = (int64_t)(mix64((uint64_t)k) & (uint64_t)(V->mcap - 1));
  while (V->mkeys[s] != -1) {
    if (V->mkeys[s] == k) return V->mvals[s];
    s = (s + 1) & (V->mcap - 1);
  }
  return -1;
}

static int insert_block(ovol* V, int x, int y, int z) {
  int b = find_block(V, x, y, z);
  if (b >= 0) return b;
  oblock* B = (oblock*)calloc(1, sizeof(oblock));
  B->key[0] = x; B->key[1] = y; B->key[2] = z;
  B->alive = 1;
  if (V->nblocks == V->bcap) {
    V->bcap = V->bcap ? V->bcap * 2 : 256;
    V->blocks = (oblock**)realloc(V->blocks, sizeof(oblock*) * (size_t)V->bcap);
  }
  b = V->nblocks++;
  V->blocks[b] = B;
  if ((V->mcount + 1) * 2 > V->mcap) {
    map_rebuild(V, V->mcap * 2);
  } else {
    int64_t k = pack_block(x, y, z);
    int64_t s = (int64_t)(mix64((uint64_t)k) & (uint64_t)(V->mcap - 1));
    while (V->mkeys[s] != -1) s = (s + 1) & (V->mcap - 1);
    V->mkeys[s] = k;
    V->mvals[s] = b;
    V->mcount++;
  }
  return b;
}

/* voxel value at global voxel g; returns 1 if the voxel is usable (allocated, W > 0) */
static int voxel_at(const ovol* V, int gx, int gy, int gz, real* d, real* w) {
  int bx = floordiv8(gx), by = floordiv8(gy), bz = floordiv8(gz);
  int b = find_block(V, bx, by, bz);
  if (b < 0) return 0;
  const oblock* B = V->blocks[b];
  int i = (gx - 8 * bx) + 8 * (gy - 8 * by) + 64 * (gz - 8 * bz);
  if (d) *d = B->tsdf[i];
  if (w) *w = B->weight[i];
  return B->weight[i] > 0;
}

/* ------------------------------------------------------------ public: lifetime */
void* or_create(double voxel_size, double trunc, double eps_refine, double w_max) {
  ensure_table();
  ovol* V = (ovol*)calloc(1, sizeof(ovol));
  V->l = (real)voxel_size;
  V->mu = (real)trunc;
  V->eps = (real)eps_refine;
  V->wmax = (real)w_max;
  V->frame = 0;
  V->epoch = 1;
  map_rebuild(V, 1024);
  return V;
}

static void free_mesh(ovol* V) {
  free(V->vkeys); free(V->vpos); free(V->vnrm); free(V->tkeys);
  V->vkeys = NULL; V->vpos = V->vnrm = NULL; V->tkeys = NULL;
  V->nv = V->nt = 0;
}

void or_destroy(void* h) {
  ovol* V = (ovol*)h;
  if (!V) return;
  for (int b = 0; b < V->nblocks; ++b) free(V->blocks[b]);
  free(V->blocks); free(V->mkeys); free(V->mvals);
  free(V->pending); free(V->last_set); free(V->frame_list);
  free(V->recs);
  free_mesh(V);
  free(V);
}

int or_table_ok(void) { ensure_table(); return table_ok; }

void or_mc_table(int* ntri, int* tris /* 256 x 5 x 3 */) {
  ensure_table();
  for (int c = 0; c < 256; ++c) {
    ntri[c] = tri_n[c];
    for (int t = 0; t < 5; ++t)
      for (int j = 0; j < 3; ++j) tris[(c * 5 + t) * 3 + j] = t < tri_n[c] ? tri_e[c][t][j] : -1;
  }
}

/* ------------------------------------------------------------ block collection (Sec. V-A, Eq. 1) */

/* 3D DDA from A to B in block-grid units: visits floor(A), then one neighbour step at a
 * time along the axis whose next cell boundary is crossed first (ties x < y < z) until
 * floor(B).  Writes up to `cap` cells; returns the number of cells on the walk. */
static int dda(const real* A, const real* B, int* out, int cap) {
  int c[3], e[3], step[3], rem[3];
  real tmax[3], tdel[3];
  for (int i = 0; i < 3; ++i) {
    c[i] = (int)floor(A[i]);
    e[i] = (int)floor(B[i]);
    real dir = B[i] - A[i];
    if (dir > 0) {
      step[i] = 1;
      tdel[i] = (real)1 / dir;
      tmax[i] = (((real)c[i] + (real)1) - A[i]) * tdel[i];
    } else if (dir < 0) {
      step[i] = -1;
      tdel[i] = (real)1 / (-dir);
      tmax[i] = (A[i] - (real)c[i]) * tdel[i];
    } else {
      step[i] = 0;
      tdel[i] = (real)INFINITY;
      tmax[i] = (real)INFINITY;
    }
    rem[i] = abs(e[i] - c[i]);
  }
  int n = 0;
  for (;;) {
    if (n < cap) { out[3 * n] = c[0]; out[3 * n + 1] = c[1]; out[3 * n + 2] = c[2]; }
    ++n;
    if (rem[0] + rem[1] + rem[2] == 0) break;
    int best = -1;
    for (int i = 0; i < 3; ++i)
      if (rem[i] > 0 && (best < 0 || tmax[i] < tmax[best])) best = i;
    c[best] += step[best];
    tmax[best] += tdel[best];
    rem[best]--;
  }
  return n;
}

int or_dda(const double* A, const double* B, int* out, int cap) {
  real a[3] = {(real)A[0], (real)A[1], (real)A[2]}, b[3] = {(real)B[0], (real)B[1], (real)B[2]};
  return dda(a, b, out, cap);
}

/* The block-grid segment of pixel (u, v) with depth D: endpoints at camera depths
 * max(D - mu, ZMIN) and D + mu on the pixel ray, mapped to world by T_wc and scaled by
 * the reciprocal of the block side 8 l.  A, B receive the endpoints in block units.
 * Divisions are taken once as reciprocals (of fx, fy, the block side) and multiplied. */
static void pixel_segment(const ovol* V, int u, int v, real D, const real* K, const real* Twc, real* A, real* B) {
  real xn = ((real)u - K[2]) * ((real)1 / K[0]);
  real yn = ((real)v - K[3]) * ((real)1 / K[1]);
  real z0 = D - V->mu;
  if (z0 < ZMIN) z0 = ZMIN;
  real z1 = D + V->mu;
  real pa[3] = {xn * z0, yn * z0, z0}, pb[3] = {xn * z1, yn * z1, z1};
  real ibs = (real)1 / (V->l * (real)BS);
  for (int i = 0; i < 3; ++i) {
    real wa = ((Twc[4 * i] * pa[0] + Twc[4 * i + 1] * pa[1]) + Twc[4 * i + 2] * pa[2]) + Twc[4 * i + 3];
    real wb = ((Twc[4 * i] * pb[0] + Twc[4 * i + 1] * pb[1]) + Twc[4 * i + 2] * pb[2]) + Twc[4 * i + 3];
    A[i] = wa * ibs;
    B[i] = wb * ibs;
  }
}

static int depth_valid(float D) { return isfinite(D) && D > 0.0f; }

/* ------------------------------------------------------------ fusion (Sec. V-A, Eq. 2) */
static void integrate_block(ovol* V, int b, const float* depth, int W, int H, const real* K, const real* Tcw) {
  oblock* B = V->blocks[b];
  for (int z = 0; z < BS; ++z)
    for (int y = 0; y < BS; ++y)
      for (int x = 0; x < BS; ++x) {
        int i = x + BS * y + BS * BS * z;
        real px = (real)(B->key[0] * BS + x) * V->l;
        real py = (real)(B->key[1] * BS + y) * V->l;
        real pz = (real)(B->key[2] * BS + z) * V->l;
        real xc = ((Tcw[0] * px + Tcw[1] * py) + Tcw[2] * pz) + Tcw[3];
        real yc = ((Tcw[4] * px + Tcw[5] * py) + Tcw[6] * pz) + Tcw[7];
        real zc = ((Tcw[8] * px + Tcw[9] * py) + Tcw[10] * pz) + Tcw[11];
        if (!(zc > 0)) continue;
        real us = ((K[0] * xc) / zc + K[2]) + (real)0.5;
        real vs = ((K[1] * yc) / zc + K[3]) + (real)0.5;
        if (!(us >= 0 && us < (real)W && vs >= 0 && vs < (real)H)) continue;
        int iu = (int)floor(us), iv = (int)floor(vs);
        float Df = depth[(size_t)iv * W + iu];
        if (!depth_valid(Df)) continue;
        real sdf = (real)Df - zc;
        if (sdf < -V->mu) continue;
        real dt = sdf < V->mu ? sdf : V->mu;
        real Wo = B->weight[i];
        if (!(sdf < V->mu)) V->stat_truncated++;
        if (V->diff_on) {
          if (V->nrec == V->rcap) {
            V->rcap = V->rcap ? 2 * V->rcap : 4096;
            V->recs = (orec*)realloc(V->recs, sizeof(orec) * (size_t)V->rcap);
          }
          orec r = {b, i, V->diff_frames, iv * W + iu, (double)Wo, (unsigned char)(sdf < V->mu)};
          V->recs[V->nrec++] = r;
        }
        real num = B->tsdf[i] * Wo + dt;
        real den = Wo + (real)1;
        B->tsdf[i] = num / den;
        B->weight[i] = den < V->wmax ? den : V->wmax;
        V->stat_voxels_integrated++;
      }
}

/* Integrate one depth frame: collect and allocate blocks (Eq. 1), then fuse (Eq. 2).
 * depth: H x W row-major float32; K = (fx, fy, cx, cy); T_wc, T_cw row-major 4x4. */
int or_integrate(void* h, const float* depth, int W, int H, const double* intr, const double* Twc_d,
                 const double* Tcw_d) {
  ovol* V = (ovol*)h;
  real K[4], Twc[16], Tcw[16];
  for (int i = 0; i < 4; ++i) K[i] = (real)intr[i];
  for (int i = 0; i < 16; ++i) Twc[i] = (real)Twc_d[i], Tcw[i] = (real)Tcw_d[i];
  V->frame++;
  if (V->advance_pending) { V->epoch++; V->advance_pending = 0; }
  V->nframe = 0;
  int cap = 64;
  int* cells = (int*)malloc(sizeof(int) * 3 * (size_t)cap);
  for (int v = 0; v < H; ++v)
    for (int u = 0; u < W; ++u) {
      float Df = depth[(size_t)v * W + u];
      if (!depth_valid(Df)) continue;
      real A[3], B[3];
      pixel_segment(V, u, v, (real)Df, K, Twc, A, B);
      int ok = 1;
      for (int i = 0; i < 3; ++i)
        if (!isfinite(A[i]) || !isfinite(B[i]) || fabs((double)A[i]) > KEY_LIM || fabs((double)B[i]) > KEY_LIM) ok = 0;
      if (!ok) continue;
      int n = dda(A, B, cells, cap);
      if (n > cap) {
        cap = n;
        cells = (int*)realloc(cells, sizeof(int) * 3 * (size_t)cap);
        dda(A, B, cells, cap);
      }
      V->stat_cells += n;
      for (int j = 0; j < n; ++j) {
        int b = insert_block(V, cells[3 * j], cells[3 * j + 1], cells[3 * j + 2]);
        oblock* Bk = V->blocks[b];
        if (Bk->touch_stamp != V->frame) {
          Bk->touch_stamp = V->frame;
          push_int(&V->frame_list, &V->nframe, &V->fcap, b);
        }
        if (Bk->touch_epoch != V->epoch) {
          Bk->touch_epoch = V->epoch;
          push_int(&V->pending, &V->npending, &V->pcap, b);
        }
      }
    }
  free(cells);
  for (int j = 0; j < V->nframe; ++j) integrate_block(V, V->frame_list[j], depth, W, H, K, Tcw);
  if (V->diff_on) V->diff_frames++;
  return 0;
}

/* ------------------------------------------------------------ cube types (Sec. V-B) and refinement (Sec. V-F) */
static int cube_code(const ovol* V, const oblock* B, int x, int y, int z, real* dv) {
  int code = 0;
  for (int k = 0; k < 8; ++k) {
    real d, w;
    int gx = B->key[0] * BS + x + CORNER[k][0];
    int gy = B->key[1] * BS + y + CORNER[k][1];
    int gz = B->key[2] * BS + z + CORNER[k][2];
    if (!voxel_at(V, gx, gy, gz, &d, &w)) return -1;
    dv[k] = d;
    if (d < 0) code |= 1 << k;
  }
  return code;
}

static int popcount8(int x) {
  int n = 0;
  for (int i = 0; i < 8; ++i) n += (x >> i) & 1;
  return n;
}

/* Eqs. 3-5: snap a disturbed raw type to the nearest admissible regular type. */
static int refine_code(int raw, int prev, const real* dv, real eps) {
  if (popcount8(raw ^ prev) > 3) return raw;
  int best = -1, bestd = 99;
  for (int j = 0; j < 6; ++j) {
    int diff = raw ^ REGULAR[j];
    int dh = popcount8(diff);
    if (dh > 3) continue;
    int ok = 1;
    for (int k = 0; k < 8; ++k)
      if (((diff >> k) & 1) && !(fabs((double)dv[k]) < (double)eps)) ok = 0;
    if (ok && dh < bestd) { best = j; bestd = dh; }
  }
  return best >= 0 ? REGULAR[best] : raw;
}

int or_refine_code(int raw, int prev, const double* d8, double eps) {
  real dv[8];
  for (int k = 0; k < 8; ++k) dv[k] = (real)d8[k];
  return refine_code(raw, prev, dv, (real)eps);
}

static const int LOWER[7][3] = {{-1, 0, 0}, {0, -1, 0}, {-1, -1, 0}, {0, 0, -1}, {-1, 0, -1}, {0, -1, -1}, {-1, -1, -1}};

/* The update set: full -> all live blocks; else the blocks collected since the last
 * mesh update and their existing lower neighbours. */
static void build_update_set(ovol* V, int full) {
  V->nlast = 0;
  for (int b = 0; b < V->nblocks; ++b) V->blocks[b]->mark = 0;
  if (full) {
    for (int b = 0; b < V->nblocks; ++b)
      if (V->blocks[b]->alive) push_int(&V->last_set, &V->nlast, &V->lcap, b);
    return;
  }
  for (int j = 0; j < V->npending; ++j) {
    oblock* B = V->blocks[V->pending[j]];
    if (!B->alive) continue;
    if (!B->mark) { B->mark = 1; push_int(&V->last_set, &V->nlast, &V->lcap, V->pending[j]); }
    for (int o = 0; o < 7; ++o) {
      int n = find_block(V, B->key[0] + LOWER[o][0], B->key[1] + LOWER[o][1], B->key[2] + LOWER[o][2]);
      if (n >= 0 && !V->blocks[n]->mark) { V->blocks[n]->mark = 1; push_int(&V->last_set, &V->nlast, &V->lcap, n); }
    }
  }
}

/* Mesh update (Secs. V-B..V-D): recompute the effective types of every cube of the
 * update set; the previous effective type is kept as t_{i-1}.  refine != 0 applies
 * Eqs. 3-5 in the same pass. */
int or_update_mesh(void* h, int full, int refine) {
  ovol* V = (ovol*)h;
  build_update_set(V, full);
  for (int j = 0; j < V->nlast; ++j) {
    oblock* B = V->blocks[V->last_set[j]];
    for (int z = 0; z < BS; ++z)
      for (int y = 0; y < BS; ++y)
        for (int x = 0; x < BS; ++x) {
          int i = x + BS * y + BS * BS * z;
          real dv[8];
          int raw = cube_code(V, B, x, y, z, dv);
          int prev = B->code_eff[i];
          int e = raw < 0 ? 0 : raw;
          if (refine && raw >= 0) e = refine_code(raw, prev, dv, V->eps);
          B->code_prev[i] = (unsigned char)prev;
          B->code_eff[i] = (unsigned char)e;
        }
  }
  V->npending = 0;
  V->advance_pending = 1;
  return 0;
}

/* Refinement pass (Sec. V-F) over the last update set (or all blocks). */
int or_refine_mesh(void* h, int full) {
  ovol* V = (ovol*)h;
  int n = full ? V->nblocks : V->nlast;
  for (int j = 0; j < n; ++j) {
    oblock* B = V->blocks[full ? j : V->last_set[j]];
    if (!B->alive) continue;
    for (int z = 0; z < BS; ++z)
      for (int y = 0; y < BS; ++y)
        for (int x = 0; x < BS; ++x) {
          int i = x + BS * y + BS * BS * z;
          real dv[8];
          int raw = cube_code(V, B, x, y, z, dv);
          B->code_eff[i] = (unsigned char)(raw < 0 ? 0 : refine_code(raw, B->code_prev[i], dv, V->eps));
        }
  }
  return 0;
}

/* ------------------------------------------------------------ garbage collection (Sec. V-E) */
static int block_has_triangles(const oblock* B) {
  for (int i = 0; i < BV; ++i)
    if (tri_n[B->code_eff[i]] > 0) return 1;
  return 0;
}

/* 1 if some live triangle (of any cube) uses an edge owned by a voxel of block B. */
static int block_owns_referenced_edge(const ovol* V, const oblock* B) {
  /* a triangle on an edge owned by voxel g lies in a cube g - o, o in {0,1}^3, so only
   * cubes of B and of its lower neighbours can reference edges owned by B */
  for (int o = -1; o < 7; ++o) {
    int nb[3] = {B->key[0], B->key[1], B->key[2]};
    if (o >= 0) { nb[0] += LOWER[o][0]; nb[1] += LOWER[o][1]; nb[2] += LOWER[o][2]; }
    int n = find_block(V, nb[0], nb[1], nb[2]);
    if (n < 0) continue;
    const oblock* C = V->blocks[n];
    for (int i = 0; i < BV; ++i) {
      int e = C->code_eff[i];
      for (int t = 0; t < tri_n[e]; ++t)
        for (int j = 0; j < 3; ++j) {
          int k = tri_e[e][t][j];
          const int* off = CORNER[EDGE[k][0]];
          int g[3] = {C->key[0] * BS + (i % 8) + off[0], C->key[1] * BS + ((i / 8) % 8) + off[1],
                      C->key[2] * BS + (i / 64) + off[2]};
          if (floordiv8(g[0]) == B->key[0] && floordiv8(g[1]) == B->key[1] && floordiv8(g[2]) == B->key[2]) return 1;
        }
    }
  }
  return 0;
}

int or_gc(void* h) {
  ovol* V = (ovol*)h;
  int* kill = (int*)calloc((size_t)(V->nblocks > 0 ? V->nblocks : 1), sizeof(int));
  int nk = 0;
  /* Before the collected blocks are meshed, the pending update set (collected blocks and
   * their lower neighbours) is kept whole; after a mesh update the update set is done with
   * and emptied here. */
  const int consumed = V->advance_pending;
  for (int b = 0; b < V->nblocks; ++b) V->blocks[b]->mark = 0;
  if (!consumed)
    for (int j = 0; j < V->npending; ++j) {
      oblock* P = V->blocks[V->pending[j]];
      P->mark = 1;
      for (int o = 0; o < 7; ++o) {
        int n = find_block(V, P->key[0] + LOWER[o][0], P->key[1] + LOWER[o][1], P->key[2] + LOWER[o][2]);
        if (n >= 0) V->blocks[n]->mark = 1;
      }
    }
  for (int b = 0; b < V->nblocks; ++b) {
    oblock* B = V->blocks[b];
    if (!B->alive || B->touch_epoch == V->epoch) continue;
    if (!consumed && B->mark) continue;
    if (block_has_triangles(B)) continue;
    int near = 0;
    for (int i = 0; i < BV && !near; ++i)
      if (B->weight[i] > 0 && B->tsdf[i] < V->mu) near = 1;
    if (near) continue;
    int lower_tri = 0;
    for (int o = 0; o < 7 && !lower_tri; ++o) {
      int n = find_block(V, B->key[0] + LOWER[o][0], B->key[1] + LOWER[o][1], B->key[2] + LOWER[o][2]);
      if (n >= 0 && block_has_triangles(V->blocks[n])) lower_tri = 1;
    }
    if (lower_tri) continue;
    if (block_owns_referenced_edge(V, B)) continue;
    kill[b] = 1;
    ++nk;
  }
  for (int b = 0; b < V->nblocks; ++b)
    if (kill[b]) V->blocks[b]->alive = 0;
  free(kill);
  if (consumed) V->nlast = 0;
  if (nk) {
    /* compact the pending and last-update lists, then the map */
    int n = 0;
    for (int j = 0; j < V->npending; ++j)
      if (V->blocks[V->pending[j]]->alive) V->pending[n++] = V->pending[j];
    V->npending = n;
    n = 0;
    for (int j = 0; j < V->nlast; ++j)
      if (V->blocks[V->last_set[j]]->alive) V->last_set[n++] = V->last_set[j];
    V->nlast = n;
    map_rebuild(V, V->mcap);
  }
  return nk;
}

/* ------------------------------------------------------------ analytic fills (tests) */
/* Allocate the blocks `keys` (n x 3) and set their voxels from tsdf/weight (n x 512 each). */
int or_set_blocks(void* h, const int* keys, int n, const double* tsdf, const double* weight) {
  ovol* V = (ovol*)h;
  for (int j = 0; j < n; ++j) {
    int b = insert_block(V, keys[3 * j], keys[3 * j + 1], keys[3 * j + 2]);
    oblock* B = V->blocks[b];
    for (int i = 0; i < BV; ++i) {
      B->tsdf[i] = (real)tsdf[(size_t)j * BV + i];
      B->weight[i] = (real)weight[(size_t)j * BV + i];
    }
    if (B->touch_epoch != V->epoch) {
      B->touch_epoch = V->epoch;
      push_int(&V->pending, &V->npending, &V->pcap, b);
    }
  }
  return 0;
}

/* ------------------------------------------------------------ exports */
int or_num_blocks(void* h) {
  ovol* V = (ovol*)h;
  int n = 0;
  for (int b = 0; b < V->nblocks; ++b) n += V->blocks[b]->alive;
  return n;
}

void or_export_blocks(void* h, int* keys, double* tsdf, double* weight, unsigned char* code_eff,
                      unsigned char* code_prev) {
  ovol* V = (ovol*)h;
  int n = 0;
  for (int b = 0; b < V->nblocks; ++b) {
    const oblock* B = V->blocks[b];
    if (!B->alive) continue;
    memcpy(keys + 3 * n, B->key, 3 * sizeof(int));
    for (int i = 0; i < BV; ++i) {
      if (tsdf) tsdf[(size_t)n * BV + i] = (double)B->tsdf[i];
      if (weight) weight[(size_t)n * BV + i] = (double)B->weight[i];
    }
    if (code_eff) memcpy(code_eff + (size_t)n * BV, B->code_eff, BV);
    if (code_prev) memcpy(code_prev + (size_t)n * BV, B->code_prev, BV);
    ++n;
  }
}

void or_stats(void* h, int64_t* out) {
  ovol* V = (ovol*)h;
  out[0] = V->stat_cells;
  out[1] = V->stat_voxels_integrated;
  out[2] = V->nframe;
  out[3] = V->nlast;
  out[4] = V->epoch;
  out[5] = V->stat_truncated;
}

/* edge key: voxel coordinates biased by 2^19 (20 bits each) and the axis (2 bits) */
static uint64_t edge_key(int gx, int gy, int gz, int axis) {
  return ((uint64_t)(gx + (1 << 19)) << 42) | ((uint64_t)(gy + (1 << 19)) << 22) | ((uint64_t)(gz + (1 << 19)) << 2) |
         (uint64_t)axis;
}

static int cmp_u64(const void* a, const void* b) {
  uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
  return (x > y) - (x < y);
}

/* Vertex of an owned edge (Sec. V-C): position and trilinear-gradient normal. */
static void edge_vertex(const ovol* V, uint64_t key, double* pos, double* nrm) {
  int g[3] = {(int)((key >> 42) & 0xFFFFF) - (1 << 19), (int)((key >> 22) & 0xFFFFF) - (1 << 19),
              (int)((key >> 2) & 0xFFFFF) - (1 << 19)};
  int a = (int)(key & 3);
  int g1[3] = {g[0], g[1], g[2]};
  g1[a] += 1;
  real d0 = 0, d1 = 0;
  voxel_at(V, g[0], g[1], g[2], &d0, NULL);
  voxel_at(V, g1[0], g1[1], g1[2], &d1, NULL);
  real t = d0 == d1 ? (real)0.5 : d0 / (d0 - d1);
  if (t < (real)-1) t = (real)-1;
  if (t > (real)2) t = (real)2;
  real p[3];
  for (int i = 0; i < 3; ++i) p[i] = (real)g[i] * V->l;
  p[a] = (real)g[a] * V->l + t * V->l;
  real n[3];
  for (int b = 0; b < 3; ++b) {
    if (b == a) { n[b] = d1 - d0; continue; }
    real e0, e1;
    int h0 = voxel_at(V, g[0] + (b == 0), g[1] + (b == 1), g[2] + (b == 2), &e0, NULL);
    int h1 = voxel_at(V, g1[0] + (b == 0), g1[1] + (b == 1), g1[2] + (b == 2), &e1, NULL);
    n[b] = (h0 && h1) ? ((real)1 - t) * (e0 - d0) + t * (e1 - d1) : (real)0;
  }
  real len = real_sqrt((n[0] * n[0] + n[1] * n[1]) + n[2] * n[2]);
  for (int i = 0; i < 3; ++i) {
    pos[i] = (double)p[i];
    nrm[i] = len > 0 ? (double)(n[i] / len) : 0.0;
  }
}

/* Build the mesh of all cubes' effective types: triangles as edge-key triples in
 * emission order and the unique vertices (sorted by key) with positions and normals.
 * Returns the vertex count; *ntri receives the triangle count. */
int64_t or_mesh_build(void* h, int64_t* ntri) {
  ovol* V = (ovol*)h;
  free_mesh(V);
  int64_t nt = 0;
  for (int b = 0; b < V->nblocks; ++b) {
    if (!V->blocks[b]->alive) continue;
    for (int i = 0; i < BV; ++i) nt += tri_n[V->blocks[b]->code_eff[i]];
  }
  V->tkeys = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(3 * nt + 1));
  int64_t k = 0;
  for (int b = 0; b < V->nblocks; ++b) {
    const oblock* B = V->blocks[b];
    if (!B->alive) continue;
    for (int i = 0; i < BV; ++i) {
      int e = B->code_eff[i];
      int cg[3] = {B->key[0] * BS + i % 8, B->key[1] * BS + (i / 8) % 8, B->key[2] * BS + i / 64};
      for (int t = 0; t < tri_n[e]; ++t)
        for (int j = 0; j < 3; ++j) {
          int ek = tri_e[e][t][j];
          const int* off = CORNER[EDGE[ek][0]];
          V->tkeys[k++] = edge_key(cg[0] + off[0], cg[1] + off[1], cg[2] + off[2], edge_axis(ek));
        }
    }
  }
  uint64_t* sorted = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(3 * nt + 1));
  memcpy(sorted, V->tkeys, sizeof(uint64_t) * (size_t)(3 * nt));
  qsort(sorted, (size_t)(3 * nt), sizeof(uint64_t), cmp_u64);
  int64_t nv = 0;
  for (int64_t j = 0; j < 3 * nt; ++j)
    if (j == 0 || sorted[j] != sorted[j - 1]) sorted[nv++] = sorted[j];
  V->vkeys = sorted;
  V->vpos = (double*)malloc(sizeof(double) * (size_t)(3 * nv + 1));
  V->vnrm = (double*)malloc(sizeof(double) * (size_t)(3 * nv + 1));
  for (int64_t j = 0; j < nv; ++j) edge_vertex(V, V->vkeys[j], V->vpos + 3 * j, V->vnrm + 3 * j);
  V->nv = nv;
  V->nt = nt;
  *ntri = nt;
  return nv;
}

void or_mesh_fetch(void* h, uint64_t* vkeys, double* pos, double* nrm, uint64_t* tkeys) {
  ovol* V = (ovol*)h;
  if (vkeys) memcpy(vkeys, V->vkeys, sizeof(uint64_t) * (size_t)V->nv);
  if (pos) memcpy(pos, V->vpos, sizeof(double) * (size_t)(3 * V->nv));
  if (nrm) memcpy(nrm, V->vnrm, sizeof(double) * (size_t)(3 * V->nv));
  if (tkeys) memcpy(tkeys, V->tkeys, sizeof(uint64_t) * (size_t)(3 * V->nt));
}

/* ------------------------------------------------------------ differentiable path */
/* Start recording integrations (and clear dL/dd).  No gc may run until the gradients
 * have been taken: block indices name the recorded voxels. */
void or_diff_begin(void* h) {
  ovol* V = (ovol*)h;
  V->diff_on = 1;
  V->diff_frames = 0;
  V->nrec = 0;
  for (int b = 0; b < V->nblocks; ++b) memset(V->blocks[b]->gd, 0, sizeof(V->blocks[b]->gd));
}

void or_diff_end(void* h) {
  ovol* V = (ovol*)h;
  V->diff_on = 0;
}

int or_diff_frames(void* h) { return ((ovol*)h)->diff_frames; }

/* dL/dd of global voxel g, or NULL when its block is not allocated */
static double* grad_at(ovol* V, int gx, int gy, int gz) {
  int bx = floordiv8(gx), by = floordiv8(gy), bz = floordiv8(gz);
  int b = find_block(V, bx, by, bz);
  if (b < 0) return NULL;
  return &V->blocks[b]->gd[(gx - 8 * bx) + 8 * (gy - 8 * by) + 64 * (gz - 8 * bz)];
}

/* Add the TSDF-value gradients of the vertices `keys` (n edge keys) given dL/dp and
 * dL/dn (n x 3 each) at their positions and normals (Sec. V-C as above):
 *   p_a = g_a l + t l, t = d0 / (d0 - d1): dt/dd0 = -d1 / (d0 - d1)^2, dt/dd1 = d0 / (d0 - d1)^2
 *   (0 where t is clamped or d0 = d1);
 *   n = m / |m|, m_a = d1 - d0, m_b = (1 - t)(e0_b - d0) + t (e1_b - d1) for b != a with
 *   both corners usable: dL/dm = (dL/dn - n (n . dL/dn)) / |m| (0 when |m| = 0). */
void or_grad_vertices(void* h, int64_t n, const uint64_t* keys, const double* gpos, const double* gnrm) {
  ovol* V = (ovol*)h;
  for (int64_t j = 0; j < n; ++j) {
    uint64_t key = keys[j];
    int g[3] = {(int)((key >> 42) & 0xFFFFF) - (1 << 19), (int)((key >> 22) & 0xFFFFF) - (1 << 19),
                (int)((key >> 2) & 0xFFFFF) - (1 << 19)};
    int a = (int)(key & 3);
    int g1[3] = {g[0], g[1], g[2]};
    g1[a] += 1;
    double* G0 = grad_at(V, g[0], g[1], g[2]);
    double* G1 = grad_at(V, g1[0], g1[1], g1[2]);
    if (!G0 || !G1) continue;
    real d0r = 0, d1r = 0;
    voxel_at(V, g[0], g[1], g[2], &d0r, NULL);
    voxel_at(V, g1[0], g1[1], g1[2], &d1r, NULL);
    real tr = d0r == d1r ? (real)0.5 : d0r / (d0r - d1r);
    const int fixed_t = d0r == d1r || tr < (real)-1 || tr > (real)2;
    if (tr < (real)-1) tr = (real)-1;
    if (tr > (real)2) tr = (real)2;
    const double d0 = (double)d0r, d1 = (double)d1r, t = (double)tr;
    double dt0 = 0, dt1 = 0;
    if (!fixed_t) {
      const double q = d0 - d1;
      dt0 = -d1 / (q * q);
      dt1 = d0 / (q * q);
    }
    double gt = gpos[3 * j + a] * (double)V->l;
    /* the normal: corner values, usability (decided as in the forward), m in float64 */
    double m[3], e0v[3] = {0, 0, 0}, e1v[3] = {0, 0, 0};
    double *GE0[3] = {NULL, NULL, NULL}, *GE1[3] = {NULL, NULL, NULL};
    real mr[3];
    int use[3] = {0, 0, 0};
    for (int b = 0; b < 3; ++b) {
      if (b == a) {
        m[b] = d1 - d0;
        mr[b] = d1r - d0r;
        continue;
      }
      real e0r = 0, e1r = 0;
      int h0 = voxel_at(V, g[0] + (b == 0), g[1] + (b == 1), g[2] + (b == 2), &e0r, NULL);
      int h1 = voxel_at(V, g1[0] + (b == 0), g1[1] + (b == 1), g1[2] + (b == 2), &e1r, NULL);
      use[b] = h0 && h1;
      if (use[b]) {
        e0v[b] = (double)e0r;
        e1v[b] = (double)e1r;
        GE0[b] = grad_at(V, g[0] + (b == 0), g[1] + (b == 1), g[2] + (b == 2));
        GE1[b] = grad_at(V, g1[0] + (b == 0), g1[1] + (b == 1), g1[2] + (b == 2));
        m[b] = (1 - t) * (e0v[b] - d0) + t * (e1v[b] - d1);
        mr[b] = ((real)1 - tr) * (e0r - d0r) + tr * (e1r - d1r);
      } else {
        m[b] = 0;
        mr[b] = 0;
      }
    }
    double gm[3] = {0, 0, 0};
    const real lenr = real_sqrt((mr[0] * mr[0] + mr[1] * mr[1]) + mr[2] * mr[2]);
    const double len = sqrt(m[0] * m[0] + m[1] * m[1] + m[2] * m[2]);
    if (lenr > 0 && len > 0) {
      double nh[3] = {m[0] / len, m[1] / len, m[2] / len};
      double dot = nh[0] * gnrm[3 * j] + nh[1] * gnrm[3 * j + 1] + nh[2] * gnrm[3 * j + 2];
      for (int i = 0; i < 3; ++i) gm[i] = (gnrm[3 * j + i] - nh[i] * dot) / len;
    }
    double gd0 = -gm[a], gd1 = gm[a];
    for (int b = 0; b < 3; ++b) {
      if (b == a || !use[b]) continue;
      *GE0[b] += gm[b] * (1 - t);
      *GE1[b] += gm[b] * t;
      gd0 -= gm[b] * (1 - t);
      gd1 -= gm[b] * t;
      gt += gm[b] * ((e1v[b] - d1) - (e0v[b] - d0));
    }
    gd0 += gt * dt0;
    gd1 += gt * dt1;
    *G0 += gd0;
    *G1 += gd1;
  }
}

/* dL/dd of every allocated block, in the order of or_export_blocks (n_blocks x 512). */
void or_grad_export(void* h, double* out) {
  ovol* V = (ovol*)h;
  int n = 0;
  for (int b = 0; b < V->nblocks; ++b) {
    if (!V->blocks[b]->alive) continue;
    memcpy(out + (size_t)n * BV, V->blocks[b]->gd, sizeof(double) * BV);
    ++n;
  }
}

/* Reverse-mode through the recorded integrations, last to first: dL/dD of every recorded
 * frame into gdepth (frames x H x W, zeroed here).  Consumes dL/dd (afterwards it holds
 * the gradient with respect to the values before the first recorded frame). */
void or_grad_depth(void* h, int W, int H, double* gdepth) {
  ovol* V = (ovol*)h;
  memset(gdepth, 0, sizeof(double) * (size_t)V->diff_frames * (size_t)W * (size_t)H);
  for (int64_t r = V->nrec - 1; r >= 0; --r) {
    const orec* R = &V->recs[r];
    double* g = &V->blocks[R->block]->gd[R->voxel];
    const double gdt = *g / (R->wpre + 1);
    if (R->lin) gdepth[(size_t)R->frame * (size_t)W * (size_t)H + (size_t)R->pixel] += gdt;
    *g = *g * R->wpre / (R->wpre + 1);
  }
}

/* Overwrite the TSDF value of one allocated voxel (finite-difference tests); 0 if absent. */
int or_set_voxel(void* h, int gx, int gy, int gz, double d) {
  ovol* V = (ovol*)h;
  int bx = floordiv8(gx), by = floordiv8(gy), bz = floordiv8(gz);
  int b = find_block(V, bx, by, bz);
  if (b < 0) return 0;
  V->blocks[b]->tsdf[(gx - 8 * bx) + 8 * (gy - 8 * by) + 64 * (gz - 8 * bz)] = (real)d;
  return 1;
}

/* ------------------------------------------------------------ mesh memory (Sec. VI-B) */
/* Vertex counts of meshes that share fewer vertices, from the effective types: out[0] the
 * distinct edges used over all blocks (this mesh), out[1] the sum over blocks of the
 * distinct edges used by each block's own cubes (a per-block extraction), out[2] three per
 * triangle (loose triangles), out[3] the triangles. */
void or_mesh_memory(void* h, int64_t* out) {
  ovol* V = (ovol*)h;
  int64_t total = 0, per_block = 0, ntri = 0;
  uint64_t* all = NULL;
  int64_t nall = 0, call = 0;
  uint64_t* loc = (uint64_t*)malloc(sizeof(uint64_t) * BV * 15);
  for (int b = 0; b < V->nblocks; ++b) {
    const oblock* B = V->blocks[b];
    if (!B->alive) continue;
    int64_t nloc = 0;
    for (int i = 0; i < BV; ++i) {
      int e = B->code_eff[i];
      int cg[3] = {B->key[0] * BS + i % 8, B->key[1] * BS + (i / 8) % 8, B->key[2] * BS + i / 64};
      ntri += tri_n[e];
      for (int t = 0; t < tri_n[e]; ++t)
        for (int j = 0; j < 3; ++j) {
          int ek = tri_e[e][t][j];
          const int* off = CORNER[EDGE[ek][0]];
          loc[nloc++] = edge_key(cg[0] + off[0], cg[1] + off[1], cg[2] + off[2], edge_axis(ek));
        }
    }
    qsort(loc, (size_t)nloc, sizeof(uint64_t), cmp_u64);
    for (int64_t j = 0; j < nloc; ++j) {
      if (j > 0 && loc[j] == loc[j - 1]) continue;
      ++per_block;
      if (nall == call) {
        call = call ? 2 * call : 4096;
        all = (uint64_t*)realloc(all, sizeof(uint64_t) * (size_t)call);
      }
      all[nall++] = loc[j];
    }
  }
  if (nall) qsort(all, (size_t)nall, sizeof(uint64_t), cmp_u64);
  for (int64_t j = 0; j < nall; ++j)
    if (j == 0 || all[j] != all[j - 1]) ++total;
  free(all);
  free(loc);
  out[0] = total;
  out[1] = per_block;
  out[2] = 3 * ntri;
  out[3] = ntri;
}
