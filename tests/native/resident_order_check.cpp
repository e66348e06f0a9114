// Host check of the resident engine's point order (csrc/resident_order.h): a bijection onto
// the extended tile, and the regions R(rr) and Rp(rr) of every step are prefixes of it.
#include <cstdio>
#include <vector>
#include <set>
#include "resident_order.h"
using namespace vomt;
int main() {
  long cases = 0;
  for (int TW = 1; TW <= 12; ++TW) for (int TH = 1; TH <= 12; ++TH)
  for (int mask = 0; mask < 16; ++mask) for (int R = 0; R <= 6; ++R) {
    TileFrame f{100, 100 + TW, 200, 200 + TH, mask & 1, (mask >> 1) & 1, (mask >> 2) & 1, (mask >> 3) & 1, R};
    if (R == 0 && mask) continue;
    int X0 = f.x0 - f.hL * R, X1 = f.x1 + f.hR * R, Y0 = f.y0 - f.hD * R, Y1 = f.y1 + f.hU * R;
    int NP = (X1 - X0) * (Y1 - Y0);
    if (region_count(f, R) != NP) { printf("count mismatch\n"); return 1; }
    std::set<std::pair<int,int>> seen;
    std::vector<int> dist(NP), distp(NP);
    for (int q = 0; q < NP; ++q) {
      int x, y;
      if (!onion_point(f, q, x, y)) { printf("no point q=%d\n", q); return 1; }
      if (x < X0 || x >= X1 || y < Y0 || y >= Y1) { printf("out of region\n"); return 1; }
      if (!seen.insert({x, y}).second) { printf("duplicate\n"); return 1; }
      int dl = f.x0 - x, dr = x - (f.x1 - 1), dd = f.y0 - y, du = y - (f.y1 - 1);
      int m = 0; if (dl > m) m = dl; if (dr > m) m = dr; if (dd > m) m = dd; if (du > m) m = du;
      int mp = 0; if (dl - 1 > mp) mp = dl - 1; if (dr > mp) mp = dr; if (dd - 1 > mp) mp = dd - 1; if (du > mp) mp = du;
      dist[q] = m; distp[q] = mp;
    }
    int xx, yy; if (onion_point(f, NP, xx, yy)) { printf("past end\n"); return 1; }
    for (int rr = 0; rr <= R; ++rr) {
      int nr = region_count(f, rr), nrp = region_p_count(f, rr);
      for (int q = 0; q < NP; ++q) {
        if ((dist[q] <= rr) != (q < nr)) { printf("R prefix fail TW=%d TH=%d mask=%d R=%d rr=%d q=%d\n", TW, TH, mask, R, rr, q); return 1; }
        if ((distp[q] <= rr) != (q < nrp)) { printf("Rp prefix fail TW=%d TH=%d mask=%d R=%d rr=%d q=%d\n", TW, TH, mask, R, rr, q); return 1; }
      }
    }
    ++cases;
  }
  printf("ok %ld cases\n", cases);
  return 0;
}
