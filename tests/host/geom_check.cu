// Host-side check of libwd's lattice index arithmetic: the multiply-shift
// division against '/', and the checkerboard -> coordinate decode against
// plain division, for every divisor and site of a range of lattices.
#include <cstdio>
#include <cstdlib>

#include "../../paper_0810_5365_gb300/csrc/wd_common.cuh"

int main() {
  using namespace wd;
  long long checked = 0;
  for (int d = 1; d <= 4096; d++) {
    FastDiv f = make_fastdiv(d);
    for (int n = 0; n < (1 << 16); n++) {
      if (fdiv(n, f) != n / d) { printf("FAIL d=%d n=%d\n", d, n); return 1; }
      checked++;
    }
    unsigned long long x = 0x9E3779B97F4A7C15ull * (unsigned)d;
    for (int k = 0; k < 4096; k++) {
      x ^= x << 13; x ^= x >> 7; x ^= x << 17;
      int n = (int)(x & 0x7fffffffu);
      if (k == 0) n = 0x7fffffff;
      if (fdiv(n, f) != n / d) { printf("FAIL d=%d n=%d\n", d, n); return 1; }
      checked++;
    }
  }
  const int shapes[][4] = {{2, 2, 2, 2}, {4, 6, 8, 10}, {6, 6, 6, 6}, {32, 32, 32, 64},
                           {2, 4, 2, 6}, {24, 24, 24, 48}, {8, 2, 4, 2}};
  for (auto& s : shapes) {
    Geom g = make_geom(s);
    for (int p = 0; p < 2; p++)
      for (int cb = 0; cb < g.Vh; cb++) {
        int x0, x1, x2, x3;
        cb_coords(cb, p, g, x0, x1, x2, x3);
        long long lex = x0 + (long long)s[0] * (x1 + (long long)s[1] * (x2 + (long long)s[2] * x3));
        if (((x0 + x1 + x2 + x3) & 1) != p || (lex >> 1) != cb || x0 < 0 || x0 >= s[0] ||
            x1 < 0 || x1 >= s[1] || x2 < 0 || x2 >= s[2] || x3 < 0 || x3 >= s[3]) {
          printf("FAIL coords cb=%d p=%d\n", cb, p);
          return 1;
        }
        checked++;
      }
  }
  printf("OK %lld\n", checked);
  return 0;
}
