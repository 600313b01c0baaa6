// Host driver for the clipping of the L2 prefetches (test infrastructure):
// for seeded random block regions of seeded random grids, every element run
// the kernels would prefetch lies inside the planes, and the runs cover the
// region clipped to the grid exactly, row by row and plane by plane.
// Also 3D: a block's z plane is a base offset z * nx * ny with the same plane
// stride N = nx * ny * nz.  Prints "ok <cases>" and exits 0, or the first bad
// case and exits 1.
#include <cstdio>
#include <random>
#include <vector>

#include "common.cuh"

int main() {
  std::mt19937_64 rng(12345);
  auto uni = [&](int a, int b) { return (int)std::uniform_int_distribution<int>(a, b)(rng); };
  int cases = 0;
  for (int it = 0; it < 20000; ++it) {
    const int nx = uni(1, 70), ny = uni(1, 40), nz = uni(1, 4), np = uni(1, 27);
    const long long sxy = (long long)nx * ny, N = sxy * nz;
    const int z = uni(0, nz - 1);
    const int rx = uni(0, 45), ry = uni(0, 30);
    const int x0 = uni(-rx - 5, nx + 5), y0 = uni(-ry - 5, ny + 5);
    std::vector<int> seen((size_t)(np * N), 0);
    for (int task = 0; task < np * ry; ++task) {
      long long e0 = 0, e1 = 0;
      if (!hz::plane_row_run(task, N, nx, ny, x0, rx, y0, ry, e0, e1)) continue;
      e0 += z * sxy;
      e1 += z * sxy;
      if (e0 < 0 || e1 >= np * N || e1 < e0) {
        printf("out of range: nx %d ny %d nz %d np %d x0 %d rx %d y0 %d ry %d task %d run [%lld, %lld]\n", nx, ny, nz,
               np, x0, rx, y0, ry, task, e0, e1);
        return 1;
      }
      for (long long e = e0; e <= e1; ++e) seen[(size_t)e] += 1;
    }
    for (int s = 0; s < np; ++s)
      for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
          const bool in = x >= x0 && x < x0 + rx && y >= y0 && y < y0 + ry;
          const long long e = (long long)s * N + z * sxy + (long long)y * nx + x;
          if (seen[(size_t)e] != (in ? 1 : 0)) {
            printf("coverage: nx %d ny %d np %d x0 %d rx %d y0 %d ry %d at (%d, %d, %d): %d\n", nx, ny, np, x0, rx, y0,
                   ry, s, x, y, seen[(size_t)e]);
            return 1;
          }
        }
    for (long long e = 0; e < np * N; ++e) {
      const long long zz = (e % N) / sxy;
      if (zz != z && seen[(size_t)e]) {
        printf("other z plane touched\n");
        return 1;
      }
    }
    ++cases;
  }
  printf("ok %d\n", cases);
  return 0;
}
