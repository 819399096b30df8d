// Host-side check of the learned proposal's ray layout as the library
// defines it (prop_rays, prop_ray and prop_index in air_internal.cuh): for
// every combination of the four quadrant depths up to a maximum level, every
// ray of a base pixel's proposal names a pixel below that base pixel, inside
// the proposed subtrees, that prop_index maps back to the same ray; no pixel
// is named twice; and the pixels just below each quadrant's proposed depth
// are reported as not traced. Prints "ok <rays checked>" and exits 0, or
// prints the first mismatch and exits 1.
#include <cstdio>
#include <set>
#include <tuple>

#include "air_internal.cuh"

using namespace air;

static int fail(const char *what, const int8_t *d4, long long r, int L, int i, int j) {
  std::printf("%s: depths %d %d %d %d ray %lld -> (%d, %d, %d)\n", what, d4[0], d4[1], d4[2], d4[3], r,
              L, i, j);
  return 1;
}

int main() {
  const int Lmax = 5;
  const int bi = 3, bj = 6;  // any base pixel: the layout is relative to it
  long long checked = 0;
  for (int a = 0; a <= Lmax; ++a)
    for (int b = 0; b <= Lmax; ++b)
      for (int c = 0; c <= Lmax; ++c)
        for (int e = 0; e <= Lmax; ++e) {
          const int8_t d4[4] = {(int8_t)a, (int8_t)b, (int8_t)c, (int8_t)e};
          const int dm = prop_max_depth(d4);
          const long long size = prop_rays(d4);
          long long expect = dm >= 1 ? 4 : 0;
          for (int q = 0; q < 4; ++q)
            for (int l = 2; l <= d4[q]; ++l) expect += 1LL << (2 * (l - 1));
          if (size != expect) return fail("ray count", d4, size, 0, 0, 0);
          std::set<std::tuple<int, int, int>> seen;
          for (long long r = 0; r < size; ++r) {
            int L = 0, i = 0, j = 0;
            prop_ray(d4, r, bi, bj, L, i, j);
            if (L < 1 || L > Lmax) return fail("level", d4, r, L, i, j);
            if ((i >> L) != bi || (j >> L) != bj) return fail("outside the base pixel", d4, r, L, i, j);
            const int q = ((i >> (L - 1)) & 1) + 2 * ((j >> (L - 1)) & 1);
            if (L >= 2 && L > d4[q]) return fail("deeper than proposed", d4, r, L, i, j);
            if (prop_index(d4, 0, L, i, j) != r) return fail("index", d4, r, L, i, j);
            if (!seen.insert(std::make_tuple(L, i, j)).second) return fail("twice", d4, r, L, i, j);
            ++checked;
          }
          // one level below each quadrant's proposal: not traced
          for (int q = 0; q < 4; ++q) {
            const int L = d4[q] >= 1 ? d4[q] + 1 : (dm >= 1 ? 2 : 1);
            if (L > Lmax) continue;
            const int i = ((2 * bi + (q & 1)) << (L - 1)), j = ((2 * bj + (q >> 1)) << (L - 1));
            if (prop_index(d4, 0, L, i, j) != -1) return fail("untraced pixel found", d4, -1, L, i, j);
          }
        }
  std::printf("ok %lld\n", checked);
  return 0;
}
