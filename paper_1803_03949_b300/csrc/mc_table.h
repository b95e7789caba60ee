// Host-side construction of the marching-cubes table T of Sec. V-B.
//
// T(t) lists, for each 8-bit cube type t (bit k set when corner k has d < 0), the
// triangles of the isosurface patch as triples of cube-edge ids.  It is built here from
// the definition rather than copied:
//   1. Walk each face's corner cycle counter-clockwise as seen from outside the cube.
//      Every maximal run of negative corners on the cycle gives one segment, from the
//      edge where the walk enters the run to the edge where it leaves.  On a face whose
//      diagonal corners alternate in sign this cuts the two negative corners off
//      separately, the same choice on both sides of the face, so neighbouring cubes
//      agree and the mesh is watertight; the direction puts the negative side on the
//      right of the segment seen from outside, so triangles face from negative to
//      positive TSDF.
//   2. The segments chain into closed loops over the sign-change edges.
//   3. A loop of m edges becomes m - 2 triangles fanned from its smallest edge id whose
//      fan diagonals never join two edges of a common cube face (a diagonal on a face
//      would be shared with the neighbouring cube and break the 2-manifold).
// Corner and edge numbering follow Bourke: corners (000)(100)(110)(010)(001)(101)(111)
// (011); edge k runs from the owner corner along one axis (see c_edge_owner).
#pragma once

#include <cstdint>
#include <cstring>

namespace vmk_host {

struct McTable {
  uint8_t ntri[256];
  uint8_t tri[256][15];
  uint16_t edgemask[256];
  bool ok;
};

inline void build_mc_table(McTable& T) {
  // corner coordinates
  static const int C[8][3] = {{0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0}, {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};
  // edge k: owner corner offset and axis
  static const int E[12][4] = {{0, 0, 0, 0}, {1, 0, 0, 1}, {0, 1, 0, 0}, {0, 0, 0, 1}, {0, 0, 1, 0}, {1, 0, 1, 1},
                               {0, 1, 1, 0}, {0, 0, 1, 1}, {0, 0, 0, 2}, {1, 0, 0, 2}, {1, 1, 0, 2}, {0, 1, 0, 2}};
  // face corner cycles, counter-clockwise seen from outside: -x, +x, -y, +y, -z, +z
  static const int F[6][4] = {{0, 4, 7, 3}, {1, 2, 6, 5}, {0, 1, 5, 4}, {3, 7, 6, 2}, {0, 3, 2, 1}, {4, 5, 6, 7}};

  auto corner_of = [&](int x, int y, int z) {
    for (int k = 0; k < 8; ++k)
      if (C[k][0] == x && C[k][1] == y && C[k][2] == z) return k;
    return -1;
  };
  // edge joining corners a and b (adjacent), by matching owner and axis
  auto edge_of = [&](int a, int b) {
    int lo[3], axis = -1;
    for (int i = 0; i < 3; ++i) {
      lo[i] = C[a][i] < C[b][i] ? C[a][i] : C[b][i];
      if (C[a][i] != C[b][i]) axis = i;
    }
    for (int k = 0; k < 12; ++k)
      if (E[k][3] == axis && E[k][0] == lo[0] && E[k][1] == lo[1] && E[k][2] == lo[2]) return k;
    return -1;
  };
  // two edges lie on a common face iff some coordinate plane (axis, value) holds both:
  // an edge along axis a at offset o lies on the planes (i, o_i) for i != a
  auto share_face = [&](int j, int k) {
    for (int i = 0; i < 3; ++i)
      if (i != E[j][3] && i != E[k][3] && E[j][i] == E[k][i]) return true;
    return false;
  };
  (void)corner_of;

  T.ok = true;
  for (int t = 0; t < 256; ++t) {
    int succ[12];
    int nsucc[12] = {0}, npred[12] = {0};
    for (int k = 0; k < 12; ++k) succ[k] = -1;
    for (int f = 0; f < 6; ++f) {
      const int* q = F[f];
      bool neg[4];
      for (int i = 0; i < 4; ++i) neg[i] = (t >> q[i]) & 1;
      // find each run of negative corners along the cycle
      for (int i = 0; i < 4; ++i) {
        int prev = (i + 3) & 3;
        if (!neg[i] || neg[prev]) continue;  // i starts a run
        int j = i;
        int steps = 0;
        while (neg[(j + 1) & 3] && steps < 4) { j = (j + 1) & 3; ++steps; }
        if (steps >= 3) break;  // whole face negative: no segment
        int e_in = edge_of(q[prev], q[i]);
        int e_out = edge_of(q[j], q[(j + 1) & 3]);
        succ[e_in] = e_out;
        nsucc[e_in]++;
        npred[e_out]++;
      }
    }
    uint16_t mask = 0;
    for (int k = 0; k < 12; ++k) {
      int a = E[k][0], b = E[k][1], c = E[k][2];
      int lo = corner_of(a, b, c);
      int hi = corner_of(a + (E[k][3] == 0), b + (E[k][3] == 1), c + (E[k][3] == 2));
      bool cross = ((t >> lo) & 1) != ((t >> hi) & 1);
      if (cross) mask |= (uint16_t)(1u << k);
      if (cross ? (nsucc[k] != 1 || npred[k] != 1) : (nsucc[k] || npred[k])) T.ok = false;
    }
    T.edgemask[t] = mask;
    int n = 0;
    bool seen[12] = {false};
    memset(T.tri[t], 0xFF, sizeof(T.tri[t]));
    for (int s = 0; s < 12; ++s) {
      if (succ[s] < 0 || seen[s]) continue;
      int loop[12], m = 0;
      for (int e = s; !seen[e] && m < 12; e = succ[e]) {
        seen[e] = true;
        loop[m++] = e;
      }
      int best = -1;
      for (int a = 0; a < m; ++a) {
        bool good = true;
        for (int i = 2; i <= m - 2 && good; ++i) good = !share_face(loop[a], loop[(a + i) % m]);
        if (good && (best < 0 || loop[a] < loop[best])) best = a;
      }
      if (best < 0) { T.ok = false; best = 0; }
      for (int i = 1; i + 1 < m; ++i) {
        if (n >= 5) { T.ok = false; break; }
        T.tri[t][3 * n + 0] = (uint8_t)loop[best];
        T.tri[t][3 * n + 1] = (uint8_t)loop[(best + i) % m];
        T.tri[t][3 * n + 2] = (uint8_t)loop[(best + i + 1) % m];
        ++n;
      }
    }
    T.ntri[t] = (uint8_t)n;
  }
}

}  // namespace vmk_host
