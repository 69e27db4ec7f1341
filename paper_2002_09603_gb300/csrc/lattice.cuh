// Structured-lattice helpers shared by the multigrid translation units:
// stencil offset tables, lattice index views (64-bit and 32-bit with
// invariant-divisor decoding) and the compile-time dispatch of block sizes,
// stencil kinds and launch schedules.
#pragma once
#include "common.cuh"

#include <type_traits>

namespace mhfp {
namespace {

static __constant__ signed char c_dia[25][3] = {
    {0, 0, -2}, {0, -1, -1}, {-1, 0, -1}, {0, 0, -1}, {1, 0, -1}, {0, 1, -1}, {0, -2, 0}, {-1, -1, 0}, {0, -1, 0},
    {1, -1, 0}, {-2, 0, 0},  {-1, 0, 0},  {0, 0, 0},  {1, 0, 0},  {2, 0, 0},  {-1, 1, 0}, {0, 1, 0},  {1, 1, 0},
    {0, 2, 0},  {0, -1, 1},  {-1, 0, 1},  {0, 0, 1},  {1, 0, 1},  {0, 1, 1},  {0, 0, 2}};
static __constant__ signed char c_dia_idx[125] = {
    -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 0,  -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1,
    -1, -1, -1, -1, -1, -1, -1, 1,  -1, -1, -1, 2,  3,  4,  -1, -1, -1, 5,  -1, -1, -1, -1, -1, -1, -1,
    -1, -1, 6,  -1, -1, -1, 7,  8,  9,  -1, 10, 11, 12, 13, 14, -1, 15, 16, 17, -1, -1, -1, 18, -1, -1,
    -1, -1, -1, -1, -1, -1, -1, 19, -1, -1, -1, 20, 21, 22, -1, -1, -1, 23, -1, -1, -1, -1, -1, -1, -1,
    -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, 24, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1, -1};

template <int KIND>
struct St;
template <>
struct St<ST_BOX1> {
  static constexpr int N = 27, R = 1, C = 13;
  __device__ static void off(int o, int& x, int& y, int& z) { x = o % 3 - 1; y = (o / 3) % 3 - 1; z = o / 9 - 1; }
  __device__ static int idx(int x, int y, int z) {
    if (x < -1 || x > 1 || y < -1 || y > 1 || z < -1 || z > 1) return -1;
    return (x + 1) + 3 * ((y + 1) + 3 * (z + 1));
  }
};
template <>
struct St<ST_DIAMOND2> {
  static constexpr int N = 25, R = 2, C = 12;
  __device__ static void off(int o, int& x, int& y, int& z) { x = c_dia[o][0]; y = c_dia[o][1]; z = c_dia[o][2]; }
  __device__ static int idx(int x, int y, int z) {
    if (x < -2 || x > 2 || y < -2 || y > 2 || z < -2 || z > 2) return -1;
    return c_dia_idx[(x + 2) + 5 * ((y + 2) + 5 * (z + 2))];
  }
};
template <>
struct St<ST_BOX2> {
  static constexpr int N = 125, R = 2, C = 62;
  __device__ static void off(int o, int& x, int& y, int& z) { x = o % 5 - 2; y = (o / 5) % 5 - 2; z = o / 25 - 2; }
  __device__ static int idx(int x, int y, int z) {
    if (x < -2 || x > 2 || y < -2 || y > 2 || z < -2 || z > 2) return -1;
    return (x + 2) + 5 * ((y + 2) + 5 * (z + 2));
  }
};

struct Lat {
  int Lx, Ly, Lz;
  long long N;
  __device__ void ijk(long long p, int& i, int& j, int& k) const {
    i = (int)(p % Lx);
    const long long r = p / Lx;
    j = (int)(r % Ly);
    k = (int)(r / Ly);
  }
  __device__ bool in(int i, int j, int k) const { return i >= 0 && i < Lx && j >= 0 && j < Ly && k >= 0 && k < Lz; }
  __device__ long long id(int i, int j, int k) const { return i + (long long)Lx * (j + (long long)Ly * k); }
};

Lat lat_of(const StructOp& A) { return Lat{A.Lx, A.Ly, A.Lz, A.N}; }

// ------------------------------------------------------------------ SpMV
// y = A x (or r = b - A x) on a lattice level; thread per lattice point.
template <int BS, int KIND, typename T>
__device__ __forceinline__ void spmv_body(const Lat& L, const T* __restrict__ val, const T* __restrict__ x,
                                          const T* __restrict__ b, T* __restrict__ y) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  int i, j, k;
  L.ijk(p, i, j, k);
  T acc[BS];
#pragma unroll
  for (int r = 0; r < BS; ++r) acc[r] = T(0);
#pragma unroll
  for (int o = 0; o < St<KIND>::N; ++o) {
    int dx, dy, dz;
    St<KIND>::off(o, dx, dy, dz);
    if (!L.in(i + dx, j + dy, k + dz)) continue;
    const long long q = p + dx + (long long)L.Lx * (dy + (long long)L.Ly * dz);
    const T* v = val + (long long)o * BS * BS * L.N + p;
#pragma unroll
    for (int r = 0; r < BS; ++r)
#pragma unroll
      for (int s = 0; s < BS; ++s) acc[r] += v[(long long)(r * BS + s) * L.N] * x[BS * q + s];
  }
#pragma unroll
  for (int r = 0; r < BS; ++r) y[BS * p + r] = b ? b[BS * p + r] - acc[r] : acc[r];
}

// ------------------------------------------------------- lattice helpers
// 32-bit lattice indexing for the coarse levels (see the coarse-level sweeps
// below).
struct Lat32 {
  int Lx, Ly, Lz, N, LxLy;
  Div32 dx, dy;
  __device__ __forceinline__ void ijk(unsigned p, int& i, int& j, int& k) const {
    const unsigned r = dx.div(p);
    i = (int)(p - r * (unsigned)Lx);
    k = (int)dy.div(r);
    j = (int)(r - (unsigned)k * (unsigned)Ly);
  }
};

// box index (x+2) + 5 (y+2) + 25 (z+2) of the o-th offset with |d|_1 <= 2,
// in box order (the order of stencil_offset for ST_DIAMOND2)
__host__ __device__ constexpr int dia_box(int o) { return o == 0 ? 12 : o == 1 ? 32 : o == 2 ? 36 : o == 3 ? 37 : o == 4 ? 38 : o == 5 ? 42 : o == 6 ? 52 : o == 7 ? 56 : o == 8 ? 57 : o == 9 ? 58 : o == 10 ? 60 : o == 11 ? 61 : o == 12 ? 62 : o == 13 ? 63 : o == 14 ? 64 : o == 15 ? 66 : o == 16 ? 67 : o == 17 ? 68 : o == 18 ? 72 : o == 19 ? 82 : o == 20 ? 86 : o == 21 ? 87 : o == 22 ? 88 : o == 23 ? 92 : 112; }
constexpr bool dia_table_matches_box_order() {
  int n = 0;
  for (int b = 0; b < 125; ++b) {
    const int x = b % 5 - 2, y = (b / 5) % 5 - 2, z = b / 25 - 2;
    if ((x < 0 ? -x : x) + (y < 0 ? -y : y) + (z < 0 ? -z : z) > 2) continue;
    if (dia_box(n++) != b) return false;
  }
  return n == 25;
}
static_assert(dia_table_matches_box_order(), "diamond offset table out of box order");

// compile-time offsets of each stencil kind
template <int KIND>
struct Sf;
template <>
struct Sf<ST_BOX1> {
  static constexpr int N = 27, R = 1;
  __device__ static constexpr int x(int o) { return o % 3 - 1; }
  __device__ static constexpr int y(int o) { return (o / 3) % 3 - 1; }
  __device__ static constexpr int z(int o) { return o / 9 - 1; }
};
template <>
struct Sf<ST_BOX2> {
  static constexpr int N = 125, R = 2;
  __device__ static constexpr int x(int o) { return o % 5 - 2; }
  __device__ static constexpr int y(int o) { return (o / 5) % 5 - 2; }
  __device__ static constexpr int z(int o) { return o / 25 - 2; }
};
template <>
struct Sf<ST_DIAMOND2> {
  static constexpr int N = 25, R = 2;
  __device__ static constexpr int x(int o) { return dia_box(o) % 5 - 2; }
  __device__ static constexpr int y(int o) { return (dia_box(o) / 5) % 5 - 2; }
  __device__ static constexpr int z(int o) { return dia_box(o) / 25 - 2; }
};

template <class F>
void dispatch_kind(int kind, F&& f) {
  if (kind == ST_BOX1) f(std::integral_constant<int, ST_BOX1>{});
  else if (kind == ST_DIAMOND2) f(std::integral_constant<int, ST_DIAMOND2>{});
  else f(std::integral_constant<int, ST_BOX2>{});
}

// block sizes of lattice levels: 1 (interface pressure), 3 (displacement),
// 6 (coarse displacement levels with the rigid-body modes; 27-point only)
template <class F>
void dispatch_bs(int bs, F&& f) {
  if (bs == 3) f(std::integral_constant<int, 3>{});
  else if (bs == 6) f(std::integral_constant<int, 6>{});
  else f(std::integral_constant<int, 1>{});
}

// the block sizes of M_II^(h)'s smoothed aggregation (coarsen)
template <class F>
void dispatch_bs13(int bs, F&& f) {
  if (bs == 3) f(std::integral_constant<int, 3>{});
  else f(std::integral_constant<int, 1>{});
}

// stencil kinds a block size occurs with: the displacement levels (3 or 6
// dofs per point) are 27-point lattices, the scalar interface-pressure levels
// 25-point (cells) or 125-point (coarser); other pairs are not instantiated
template <int BS, class F>
void dispatch_kind_bs(int kind, F&& f) {
  if constexpr (BS != 1) {
    if (kind != ST_BOX1) throw Error{MHFP_ERR_ARG, "vector lattice levels are 27-point only"};
    f(std::integral_constant<int, ST_BOX1>{});
  } else {
    if (kind == ST_DIAMOND2) f(std::integral_constant<int, ST_DIAMOND2>{});
    else if (kind == ST_BOX2) f(std::integral_constant<int, ST_BOX2>{});
    else throw Error{MHFP_ERR_ARG, "scalar lattice levels are 25- or 125-point"};
  }
}

// (fine, coarse) block pairs of the transfers
template <class F>
void dispatch_pair(int bf, int bc, F&& f) {
  if (bf == 3 && bc == 3) f(std::integral_constant<int, 3>{}, std::integral_constant<int, 3>{});
  else if (bf == 3 && bc == 6) f(std::integral_constant<int, 3>{}, std::integral_constant<int, 6>{});
  else if (bf == 6 && bc == 6) f(std::integral_constant<int, 6>{}, std::integral_constant<int, 6>{});
  else f(std::integral_constant<int, 1>{}, std::integral_constant<int, 1>{});
}

template <class F>
void dispatch_r(int R, F&& f) {
  if (R == 2) f(std::integral_constant<int, 2>{});
  else f(std::integral_constant<int, 1>{});
}

// 32-bit lattice view for the coarse-level kernels (their indices e N + p
// and bs q + s stay below 2^31)
inline Lat32 lat32_of(const StructOp& A) {
  if ((long long)A.bs * A.bs * A.N >= (1LL << 31))
    throw Error{MHFP_ERR_ARG, "lattice level too large for 32-bit indexing"};
  Lat32 L;
  L.Lx = A.Lx;
  L.Ly = A.Ly;
  L.Lz = A.Lz;
  L.N = (int)A.N;
  L.LxLy = A.Lx * A.Ly;
  L.dx = Div32::make((unsigned)A.Lx);
  L.dy = Div32::make((unsigned)A.Ly);
  return L;
}

// Launch schedule of a level's sweeps and residuals: 1 = one point per
// thread, W = 4, 8, 16 = warp-split offsets over W warps.  The set-up
// autotuner times all four; without it, scalar levels of 64K points and up
// take one point per thread and the others eight warps.
inline int default_schedule(long long npts, int bs) { return (bs == 1 && npts >= 65536) ? 1 : 8; }

template <class F>
void dispatch_sched(int sched, F&& f) {
  if (sched == 1) f(std::integral_constant<int, 1>{});
  else if (sched == 4) f(std::integral_constant<int, 4>{});
  else if (sched == 16) f(std::integral_constant<int, 16>{});
  else f(std::integral_constant<int, 8>{});
}

}  // namespace

// Coarse-level sweeps and residuals (sweep.cu, one object per value type):
// y = b - A x (y = A x when b is null) on a lattice level with launch
// schedule sched; one Chebyshev step from xin (see the kernels); the first
// Chebyshev step from x = 0 (no stencil work).  They queue one kernel on
// `stream` and do not check or count it: the caller does.
template <typename T>
void sweep_spmv(cudaStream_t stream, const StructOp& A, int bs, const T* val, const T* x, const T* b, T* y,
                int sched);
template <typename T>
void sweep_cheb(cudaStream_t stream, const StructOp& A, int bs, const T* val, const T* dinv, const T* b,
                const T* xin, T* out, T* d, T cd, T cr, int sched);
template <typename T>
void sweep_cheb_zero(cudaStream_t stream, long long npts, int bs, const T* dinv, const T* b, T* out, T* d, T cr);

}  // namespace mhfp
