// Precision dispatch of the V-cycle pieces (kernels in cycle_impl.cuh,
// instantiated by cycle_f32*.cu and cycle_f64*.cu).
#include "cycle_inst.cuh"

namespace hz {
namespace cyc {
HZ_CYC_ALL(extern, float)
HZ_CYC_ALL(extern, double)
}  // namespace cyc
using namespace cyc;

void level_residual(Ctx& c, int l, const void* u, const void* f, void* r, const int* active, cudaStream_t s) {
  if (c.mixed) resid<float>(c, l, u, f, r, active, s);
  else resid<double>(c, l, u, f, r, active, s);
}
void level_smooth(Ctx& c, int l, void* u, const void* f, bool u_is_zero, const int* active, cudaStream_t s) {
  if (u_is_zero) {
    if (c.mixed) sweep0<float>(c, l, f, u, active, s);
    else sweep0<double>(c, l, f, u, active, s);
    return;
  }
  level_residual(c, l, u, f, c.L[l].r, active, s);
  level_vanka_apply(c, l, c.L[l].r, u, s);
}
void level_vanka_apply(Ctx& c, int l, const void* r, void* u, cudaStream_t s) {
  if (c.mixed) sweep_out<float>(c, l, r, u, u, nullptr, s);
  else sweep_out<double>(c, l, r, u, u, nullptr, s);
}
void level_restrict(Ctx& c, int l, const void* r, void* fc, const int* active, cudaStream_t s) {
  if (c.mixed) restrict_t<float>(c, l, r, fc, active, s);
  else restrict_t<double>(c, l, r, fc, active, s);
}
void level_prolong_add(Ctx& c, int l, const void* ec, void* u, const int* active, cudaStream_t s) {
  if (c.mixed) prolong_t<float>(c, l, ec, u, u, active, s);
  else prolong_t<double>(c, l, ec, u, u, active, s);
}
void coarse_solve(Ctx& c, const void* f, void* u, const int* active, cudaStream_t s) {
  if (c.mixed) coarse_t<float>(c, f, u, active, s);
  else coarse_t<double>(c, f, u, active, s);
}
void vcycle(Ctx& c, const void* f, void* u, const int* active, cudaStream_t s) {
  if (c.mixed) vcycle_t<float>(c, 0, f, u, active, s);
  else vcycle_t<double>(c, 0, f, u, active, s);
}

namespace {
template <typename U>
__global__ void k_fine_apply64(Geo gg, int dim, double invh2, const double2* __restrict__ diag,
                               const U* __restrict__ v, double2* __restrict__ w) {
  int x, y, z, p, q;
  if (!node_xyz(gg, x, y, z, p, q)) return;
  auto ld = [v](int i) {
    const U a = v[i];
    return make_double2((double)a.x, (double)a.y);
  };
  w[q] = dim == 3 ? fine_Au<double, 3, true>(gg, invh2, diag[p], ld, q, x, y, z)
                  : fine_Au<double, 2, true>(gg, invh2, diag[p], ld, q, x, y, z);
}
// the compact fine operator in FP64 (sig = sigma per node, dsig the shift)
template <typename U>
__global__ void k_compact_apply64(GridDev gd, double invh2, const double2* __restrict__ sig, double2 dsig,
                                  const U* __restrict__ v, double2* __restrict__ w) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= gd.N) return;
  const int x = (int)(p % gd.nx);
  const long long t = p / gd.nx;
  const int y = (int)(t % gd.ny), z = (int)(t / gd.ny);
  auto ld = [v](long long q) {
    const U a = v[q];
    return make_double2((double)a.x, (double)a.y);
  };
  w[p] = compact_Av(gd.nx, gd.ny, gd.nz, gd.dim, invh2, sig, dsig, ld, p, x, y, z);
}
}  // namespace

void fine_apply_f64(Ctx& c, const void* v, bool v_single, double2* w, bool shifted, cudaStream_t s) {
  Level& L = c.L[0];
  if (c.compact) {
    require(c.nrhs == 1, "the compact stencil takes one right-hand side");
    const double2 dsig = make_double2(0.0, shifted ? -c.alpha * c.omega * c.omega : 0.0);
    const double invh2 = 1.0 / (c.h * c.h);
    if (v_single)
      k_compact_apply64<float2><<<nblk(L.g.N, 256), 256, 0, s>>>(L.g, invh2, c.diagA64, dsig, (const float2*)v, w);
    else
      k_compact_apply64<double2><<<nblk(L.g.N, 256), 256, 0, s>>>(L.g, invh2, c.diagA64, dsig, (const double2*)v, w);
    HZ_LAUNCHED();
    return;
  }
  const double2* diag = shifted ? L.A64 : c.diagA64;    // plane 0 of the FP64 fine planes is diag(A_s)
  const double invh2 = 1.0 / (c.h * c.h);
  const Geo g = geo(L.g, c.nrhs);
  if (v_single)
    k_fine_apply64<float2><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, L.g.dim, invh2, diag, (const float2*)v, w);
  else
    k_fine_apply64<double2><<<grid_of(g), dim3(BX, BY), 0, s>>>(g, L.g.dim, invh2, diag, (const double2*)v, w);
  HZ_LAUNCHED();
}

}  // namespace hz
