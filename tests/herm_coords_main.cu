// Prints the library's real-coordinate index maps (herm_coord,
// herm_pair_coord of lb_internal.cuh) for each d on the command line, for
// tests/test_herm_coords.py to compare with the oracle's coordinate order.
// Host code only: runs without a GPU.
#include <cstdio>
#include <cstdlib>

#include "lb_internal.cuh"

int main(int argc, char** argv) {
  for (int i = 1; i < argc; i++) {
    const int d = std::atoi(argv[i]);
    std::printf("d %d\n", d);
    for (int a = 0; a < d * d; a++) {
      int k, l, part;
      lb::herm_coord(a, d, &k, &l, &part);
      std::printf("c %d %d %d %d\n", a, k, l, part);
    }
    for (int k = 0; k < d; k++)
      for (int l = k + 1; l < d; l++) std::printf("p %d %d %d\n", k, l, lb::herm_pair_coord(k, l, d));
  }
  return 0;
}
