// Host driver for the integer-pipe float <-> double conversions of the CUDA
// path (test infrastructure): reads raw float32 / float64 bit patterns, writes
// f2d_exact / d2f_rn of each, for a bit-for-bit comparison with numpy.
// usage: conv_check <f32 in> <f64 out> <f64 in> <f32 out>
//        conv_check --sum <f32 in, groups of 6> <f64 out: fsum_wide of the first 4 and of all 6>
//        conv_check --pow2 <k> <f32 in> <f64 out: f2d_exact_pow2 of each value>
//        conv_check --sum-pow2 <k> <f32 in, groups of 6> <f64 out: fsum_wide_pow2 of the first 4 and of all 6>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "krylov_impl.cuh"

static int sums(const char* in, const char* out, int k = -1) {
  FILE* f = fopen(in, "rb");
  if (!f) return 3;
  std::vector<float> v;
  float x;
  while (fread(&x, 4, 1, f) == 1) v.push_back(x);
  fclose(f);
  std::vector<double> r;
  for (size_t i = 0; i + 6 <= v.size(); i += 6) {
    const float a4[4] = {v[i], v[i + 1], v[i + 2], v[i + 3]};
    const float a6[6] = {v[i], v[i + 1], v[i + 2], v[i + 3], v[i + 4], v[i + 5]};
    r.push_back(k < 0 ? hz::fsum_wide<4>(a4) : hz::fsum_wide_pow2<4>(a4, k));
    r.push_back(k < 0 ? hz::fsum_wide<6>(a6) : hz::fsum_wide_pow2<6>(a6, k));
  }
  FILE* o = fopen(out, "wb");
  if (!o) return 4;
  fwrite(r.data(), 8, r.size(), o);
  fclose(o);
  return 0;
}

static int widen_pow2(int k, const char* in, const char* out) {
  FILE* f = fopen(in, "rb");
  if (!f) return 3;
  std::vector<double> r;
  float x;
  while (fread(&x, 4, 1, f) == 1) r.push_back(hz::f2d_exact_pow2(x, k));
  fclose(f);
  FILE* o = fopen(out, "wb");
  if (!o) return 4;
  fwrite(r.data(), 8, r.size(), o);
  fclose(o);
  return 0;
}

int main(int argc, char** argv) {
  if (argc == 4 && strcmp(argv[1], "--sum") == 0) return sums(argv[2], argv[3]);
  if (argc == 5 && strcmp(argv[1], "--pow2") == 0) return widen_pow2(atoi(argv[2]), argv[3], argv[4]);
  if (argc == 5 && strcmp(argv[1], "--sum-pow2") == 0) return sums(argv[3], argv[4], atoi(argv[2]));
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
