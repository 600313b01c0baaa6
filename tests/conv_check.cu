// Host driver for the integer-pipe float <-> double conversions of the CUDA
// path (test infrastructure): reads raw float32 / float64 bit patterns, writes
// f2d_exact / d2f_rn of each, for a bit-for-bit comparison with numpy.
// usage: conv_check <f32 in> <f64 out> <f64 in> <f32 out>
#include <cstdio>
#include <vector>

#include "common.cuh"

int main(int argc, char** argv) {
  if (argc != 5) return 2;
  auto rd = [](const char* p, size_t el, std::vector<unsigned char>& b) {
    FILE* f = fopen(p, "rb");
    if (!f) return false;
    fseek(f, 0, SEEK_END);
    b.resize(ftell(f));
    fseek(f, 0, SEEK_SET);
    const bool ok = fread(b.data(), 1, b.size(), f) == b.size() && b.size() % el == 0;
    fclose(f);
    return ok;
  };
  std::vector<unsigned char> a, c;
  if (!rd(argv[1], 4, a) || !rd(argv[3], 8, c)) return 3;
  const size_t na = a.size() / 4, nc = c.size() / 8;
  std::vector<double> wide(na);
  std::vector<float> narrow(nc);
  for (size_t i = 0; i < na; ++i) {
    float f;
    memcpy(&f, &a[4 * i], 4);
    wide[i] = hz::f2d_exact(f);
  }
  for (size_t i = 0; i < nc; ++i) {
    double d;
    memcpy(&d, &c[8 * i], 8);
    narrow[i] = hz::d2f_rn(d);
  }
  FILE* o1 = fopen(argv[2], "wb");
  FILE* o2 = fopen(argv[4], "wb");
  if (!o1 || !o2) return 4;
  fwrite(wide.data(), 8, na, o1);
  fwrite(narrow.data(), 4, nc, o2);
  fclose(o1);
  fclose(o2);
  return 0;
}
