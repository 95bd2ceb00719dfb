// Host check of the grid multigrid's index arithmetic (paper_2301_01396_gb300/csrc/
// xpbd_mg_index.h), the same functions the kernels call.  Prints "ok" or the first
// violation and exits non-zero.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "xpbd_mg_index.h"

using namespace xpbd;

static int fail(const char* what, int nx, int ny, int a, int b) {
  std::printf("FAIL %s nx=%d ny=%d (%d, %d)\n", what, nx, ny, a, b);
  return 1;
}

static int check_grid(int nx, int ny) {
  const int V = nx * ny;
  // diagonal lines, both directions: every vertex on exactly one line, the line it sits on
  for (int dir = -1; dir <= 1; dir += 2) {
    std::vector<int> seen(V, 0), line_of(V, -1);
    for (int l = 0; l < nx + ny - 1; ++l) {
      int x0, y0;
      const int len = mg_line(l, nx, ny, dir, x0, y0);
      if (len < 1) return fail("empty line", nx, ny, dir, l);
      for (int k = 0; k < len; ++k) {
        const int x = x0 + dir * k, y = y0 + k;
        if (x < 0 || x >= nx || y < 0 || y >= ny) return fail("line point outside", nx, ny, l, k);
        if ((dir > 0 ? x - y + ny - 1 : x + y) != l) return fail("line point on another diagonal", nx, ny, l, k);
        seen[y * nx + x]++;
        line_of[y * nx + x] = l;
      }
    }
    for (int v = 0; v < V; ++v)
      if (seen[v] != 1) return fail("line cover", nx, ny, dir, v);
    // same-colour lines do not interact through the 5 x 5 stencil
    for (int v = 0; v < V; ++v)
      for (int dy = -2; dy <= 2; ++dy)
        for (int dx = -2; dx <= 2; ++dx) {
          const int x = v % nx + dx, y = v / nx + dy;
          if (x < 0 || x >= nx || y < 0 || y >= ny) continue;
          const int u = y * nx + x;
          if (line_of[u] != line_of[v] && line_of[u] % 5 == line_of[v] % 5)
            return fail("same-colour lines interact", nx, ny, v, u);
        }
    // the compact residual items cover each colour's vertices once
    std::vector<int> item_seen(V, 0);
    for (int c = 0; c < 5; ++c) {
      const int items = mg_line_items(nx, ny, c);
      for (int t = 0; t < items; ++t) {
        int v;
        if (!mg_line_item(t, nx, ny, dir, c, v)) continue;
        if (v < 0 || v >= V) return fail("line item outside", nx, ny, c, t);
        if (line_of[v] % 5 != c) return fail("line item of another colour", nx, ny, c, t);
        item_seen[v]++;
      }
      int lines = 0;
      for (int l = c; l < nx + ny - 1; l += 5) ++lines;
      if (lines != mg_color_lines(nx, ny, c)) return fail("colour line count", nx, ny, c, lines);
    }
    for (int v = 0; v < V; ++v)
      if (item_seen[v] != 1) return fail("line item cover", nx, ny, dir, v);
  }
  // point colours: every vertex once; same-colour vertices three cells apart
  std::vector<int> pseen(V, 0);
  for (int c = 0; c < 9; ++c) {
    const int n = mg_color_points(nx, ny, c);
    for (int t = 0; t < n; ++t) {
      const int v = mg_color_point(t, nx, c);
      if (v < 0 || v >= V) return fail("point outside", nx, ny, c, t);
      if ((v % nx) % 3 != c % 3 || (v / nx) % 3 != c / 3) return fail("point of another colour", nx, ny, c, t);
      pseen[v]++;
    }
  }
  for (int v = 0; v < V; ++v)
    if (pseen[v] != 1) return fail("point cover", nx, ny, 0, v);
  // prolongation: weights are a partition of unity, supported on the index ranges the
  // restriction ([2X-1, 2X+1]) and prolongation ((x-1)/2 .. (x+1)/2) loops visit
  for (int n : {nx, ny}) {
    const int nc = mg_coarse(n);
    for (int x = 0; x < n; ++x) {
      double s = 0.0;
      for (int X = 0; X < nc; ++X) {
        const double w = mg_w(x, X, nc);
        if (w < 0.0) return fail("negative weight", nx, ny, x, X);
        if (w != 0.0 && (x < 2 * X - 1 || x > 2 * X + 1)) return fail("weight outside restriction range", nx, ny, x, X);
        if (w != 0.0 && (X < (x - 1) / 2 || X > (x + 1) / 2)) return fail("weight outside prolongation range", nx, ny, x, X);
        s += w;
      }
      if (std::fabs(s - 1.0) > 1e-15) return fail("partition of unity", nx, ny, x, n);
    }
  }
  // workspace: the carved arrays end inside the allocation, levels end at <= 4 x 4
  for (int dir = -1; dir <= 1; ++dir) {
    const size_t words = mg_workspace_doubles(nx, ny, dir != 0);
    if (words > ((size_t)8 << 20)) continue;   // larger grids: layout as for the ones checked
    std::vector<double> buf(words);
    static MgPlan g;
    double* base = buf.data();
    double* end = mg_carve(g, base, nx, ny, dir, 1);
    size_t used = (size_t)(end - base);
    if (dir != 0) used += ((size_t)V * kMgLineFactor + 1) / 2;
    if (used != words) return fail("workspace size", nx, ny, (int)used, (int)words);
    const MgLevel& lc = g.lv[g.levels - 1];
    if (lc.nx * lc.ny > kMgCoarseMax) return fail("coarsest level too large", nx, ny, lc.nx, lc.ny);
    for (int l = 1; l < g.levels; ++l)
      if (g.lv[l].nx != mg_coarse(g.lv[l - 1].nx) || g.lv[l].ny != mg_coarse(g.lv[l - 1].ny))
        return fail("level size", nx, ny, l, g.lv[l].nx);
  }
  return 0;
}

int main() {
  int checked = 0;
  for (int nx = 1; nx <= 37; ++nx)
    for (int ny = 1; ny <= 37; ny += (ny < 12 ? 1 : 5)) {
      if (check_grid(nx, ny)) return 1;
      ++checked;
    }
  for (int n : {64, 65, 127, 128, 256}) {
    if (check_grid(n, n)) return 1;
    ++checked;
  }
  std::printf("ok %d grids\n", checked);
  return 0;
}
