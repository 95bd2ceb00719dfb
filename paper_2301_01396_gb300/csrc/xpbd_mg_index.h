// Index arithmetic of the grid multigrid (xpbd_multigrid.cuh): level sizes and workspace
// layout, bilinear prolongation weights, the grid diagonals of the line smoother and the
// colour classes of the point smoother.  Plain C++ usable from device code, so that a host
// program can check it (every vertex covered once, colours independent, weights a
// partition of unity, the workspace layout inside its allocation).
#pragma once

#include <stddef.h>

#ifdef __CUDACC__
#define XPBD_HD __host__ __device__ __forceinline__
#else
#define XPBD_HD inline
#endif

namespace xpbd {

constexpr int kMgSlots = 25;            // 5 x 5 stencil offsets
constexpr int kMgBlock = kMgSlots * 9;  // float64 per vertex of a level matrix
constexpr int kMgLineFactor = 27;       // float32 per vertex: two sub-diagonal blocks, an inverse pivot
constexpr int kMgMaxLevels = 32;        // halving any int side reaches <= 4 within 31 levels
constexpr int kMgCoarseMax = 16;        // vertices of the densely inverted level

struct MgLevel {
  int nx = 0, ny = 0;
  double* A = nullptr;     // [n][25][9]
  double* dinv = nullptr;  // [n][9] inverse diagonal blocks (zero where a row is empty or pinned)
  double* x = nullptr;     // [n][3] correction (level 0: the caller's output)
  double* b = nullptr;     // [n][3] right-hand side (level 0: the caller's input)
  double* r = nullptr;     // [n][3] residual / line-solve scratch
};

struct MgPlan {
  int levels = 0;
  MgLevel lv[kMgMaxLevels];
  double* cinv = nullptr;   // dense inverse of the coarsest level, (3 n_c)^2
  float* lfac = nullptr;    // level-0 line factors [n0][27] float32, or null without line smoothing
  int line_dir = 0;         // 0: point smoothing on level 0; +1: lines x - y = c; -1: lines x + y = c
  int sweeps = 1;
};

XPBD_HD int mg_min(int a, int b) { return a < b ? a : b; }

// Bilinear prolongation weight of coarse index X for fine index x (nc coarse points):
// fine 2X takes X; an odd fine index takes the mean of its two coarse neighbours, or the
// one it has at the far boundary.
XPBD_HD double mg_w(int x, int X, int nc) {
  const int d = x - 2 * X;
  if (d == 0) return 1.0;
  if (d == 1) return X + 1 < nc ? 0.5 : 1.0;
  if (d == -1) return 0.5;
  return 0.0;
}

// Coarse side of a fine side.
XPBD_HD int mg_coarse(int n) { return (n + 1) / 2; }

// Lines of direction dir (+1: x - y = const, -1: x + y = const), numbered 0 .. nx + ny - 2;
// point k of line l is (x0 + dir k, y0 + k); returns the line's length.
XPBD_HD int mg_line(int l, int nx, int ny, int dir, int& x0, int& y0) {
  if (dir > 0) {
    const int c = l - (ny - 1);
    y0 = c < 0 ? -c : 0;
    x0 = y0 + c;
    return mg_min(ny - y0, nx - x0);
  }
  y0 = l > nx - 1 ? l - (nx - 1) : 0;
  x0 = l - y0;
  return mg_min(ny - y0, x0 + 1);
}

// Lines of one colour (lines l = color + 5 j).
XPBD_HD int mg_color_lines(int nx, int ny, int color) { return (nx + ny - 1 - color + 4) / 5; }

// Item t of a colour's line residual: point t % L of line color + 5 (t / L), with
// L = min(nx, ny) >= every line's length.  Items = lines x L; returns false for the items
// past a line's end.
XPBD_HD int mg_line_items(int nx, int ny, int color) { return mg_color_lines(nx, ny, color) * mg_min(nx, ny); }
XPBD_HD bool mg_line_item(int t, int nx, int ny, int dir, int color, int& v) {
  const int L = mg_min(nx, ny);
  const int l = color + 5 * (t / L), k = t % L;
  if (l >= nx + ny - 1) return false;
  int x0, y0;
  if (k >= mg_line(l, nx, ny, dir, x0, y0)) return false;
  v = (y0 + k) * nx + x0 + dir * k;
  return true;
}

// Point colour c = 3 cy + cx: vertices (cx + 3 i, cy + 3 j).
XPBD_HD int mg_color_points(int nx, int ny, int color) {
  const int cx = color % 3, cy = color / 3;
  return ((nx - cx + 2) / 3) * ((ny - cy + 2) / 3);
}
XPBD_HD int mg_color_point(int t, int nx, int color) {
  const int cx = color % 3, cy = color / 3, nxs = (nx - cx + 2) / 3;
  return (cy + 3 * (t / nxs)) * nx + cx + 3 * (t % nxs);
}

// float64 count of the workspace for an nx x ny grid (levels, coarse inverse, line factors).
inline size_t mg_workspace_doubles(int nx, int ny, bool lines) {
  size_t tot = 0;
  int x = nx, y = ny, levels = 0;
  while (true) {
    const size_t n = (size_t)x * y;
    tot += n * (kMgBlock + 9 + 9);   // A, dinv, x, b, r
    ++levels;
    if ((x <= 4 && y <= 4) || levels == kMgMaxLevels) break;
    x = mg_coarse(x);
    y = mg_coarse(y);
  }
  const size_t nc3 = 3 * (size_t)x * y;
  tot += nc3 * nc3;
  if (lines) tot += ((size_t)nx * ny * kMgLineFactor + 1) / 2;   // float32 factors
  return tot;
}

// Lays the plan's arrays out in `base` (mg_workspace_doubles of them); returns the end of
// the float64 part (the line factors follow it).
inline double* mg_carve(MgPlan& g, double* base, int nx, int ny, int line_dir, int sweeps) {
  g = MgPlan();
  g.line_dir = line_dir;
  g.sweeps = sweeps;
  int x = nx, y = ny;
  double* p = base;
  while (true) {
    MgLevel& L = g.lv[g.levels++];
    const size_t n = (size_t)x * y;
    L.nx = x;
    L.ny = y;
    L.A = p;
    p += n * kMgBlock;
    L.dinv = p;
    p += 9 * n;
    L.x = p;
    p += 3 * n;
    L.b = p;
    p += 3 * n;
    L.r = p;
    p += 3 * n;
    if ((x <= 4 && y <= 4) || g.levels == kMgMaxLevels) break;
    x = mg_coarse(x);
    y = mg_coarse(y);
  }
  g.cinv = p;
  p += 9 * (size_t)x * y * x * y;
  g.lfac = line_dir ? reinterpret_cast<float*>(p) : nullptr;
  return p;
}

}  // namespace xpbd
