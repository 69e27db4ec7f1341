// Sweeps and residuals of the coarse lattice levels (displacement levels
// below the finest one, the interface-pressure cell levels), compiled once
// per value type (MHFP_SWEEP_T = float or double) so the many launch-schedule
// instantiations build in parallel.
#include "lattice.cuh"

#ifndef MHFP_SWEEP_T
#error "compile with -DMHFP_SWEEP_T=float or -DMHFP_SWEEP_T=double"
#endif

namespace mhfp {
namespace {

// ------------------------------------------------------- coarse-level sweeps
// Sweeps and residuals of the coarse lattice levels and of the interface-
// pressure cell levels.  Their data is a few to a few tens of MB, so the cost
// is latency and issue, not bytes: index arithmetic is 32-bit (the lattice
// point is split with multiply-high division by invariant integers,
// Granlund & Montgomery 1994, no 64-bit division), stencil offsets are
// compile-time constants, bounds are three small per-axis masks, and every
// offset of a chunk issues its loads before any is used (an out-of-lattice
// neighbour reads the point itself and is then replaced by 0).

// r -= sum over the offsets o with o % step == first of A(p, p + e_o) x(p + e_o)
template <int BS, int KIND, int CHUNK, typename T>
__device__ __forceinline__ void coarse_residual(const Lat32& L, unsigned p, const T* __restrict__ val,
                                                const T* __restrict__ x, T r[BS], int first, int step) {
  constexpr int R = Sf<KIND>::R, NO = Sf<KIND>::N;
  int i, j, k;
  L.ijk(p, i, j, k);
  bool mx[2 * R + 1], my[2 * R + 1], mz[2 * R + 1];
#pragma unroll
  for (int t = -R; t <= R; ++t) {
    mx[t + R] = (unsigned)(i + t) < (unsigned)L.Lx;
    my[t + R] = (unsigned)(j + t) < (unsigned)L.Ly;
    mz[t + R] = (unsigned)(k + t) < (unsigned)L.Lz;
  }
  const unsigned N = (unsigned)L.N;
#pragma unroll
  for (int o0 = 0; o0 < NO; o0 += CHUNK) {
    T vv[CHUNK][BS * BS], xx[CHUNK][BS];
#pragma unroll
    for (int c = 0; c < CHUNK; ++c) {
      const int o = o0 + c;
      if (o < NO && o % step == first) {
        const int dx = Sf<KIND>::x(o), dy = Sf<KIND>::y(o), dz = Sf<KIND>::z(o);
        const bool in = mx[dx + R] && my[dy + R] && mz[dz + R];
        const unsigned q = in ? p + (unsigned)(dx + L.Lx * dy + L.LxLy * dz) : p;
        const T* row = val + (size_t)o * BS * BS * N;
#pragma unroll
        for (int e = 0; e < BS * BS; ++e) vv[c][e] = row[e * N + p];
#pragma unroll
        for (int s = 0; s < BS; ++s) {
          const T xs = x[BS * q + s];
          xx[c][s] = in ? xs : T(0);  // a select, not a multiply (no FP64 pipe work)
        }
      }
    }
#pragma unroll
    for (int c = 0; c < CHUNK; ++c)
      if (o0 + c < NO && (o0 + c) % step == first)
#pragma unroll
        for (int a = 0; a < BS; ++a)
#pragma unroll
          for (int s = 0; s < BS; ++s) r[a] -= vv[c][a * BS + s] * xx[c][s];
  }
}

// one point per thread: loads of CHUNK offsets in flight at once
template <int BS, typename T>
constexpr int f_chunk() { return BS == 6 ? 1 : (sizeof(T) == 4 ? (BS == 1 ? 25 : 3) : (BS == 1 ? 8 : 1)); }

// y = b - A x, or y = A x when b is null
template <int BS, int KIND, typename T>
__global__ void __launch_bounds__(256) k_spmv_f(Lat32 L, const T* __restrict__ val, const T* __restrict__ x,
                                                const T* __restrict__ b, T* __restrict__ y, long long lb) {
  x = lane_ptr(x, lb);
  b = lane_ptr(b, lb);
  y = lane_ptr(y, lb);
  const unsigned p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (unsigned)L.N) return;
  T r[BS];
#pragma unroll
  for (int a = 0; a < BS; ++a) r[a] = T(0);
  coarse_residual<BS, KIND, f_chunk<BS, T>(), T>(L, p, val, x, r, 0, 1);
#pragma unroll
  for (int a = 0; a < BS; ++a) y[BS * p + a] = b ? b[BS * p + a] + r[a] : -r[a];
}

// Chebyshev step: r = b - A xin (r = b when xin is null), d = cd d + cr D^-1 r, xout = xin + d
template <typename T, int BS>
__device__ __forceinline__ void cheb_update(unsigned p, unsigned N, const T r[BS], const T* __restrict__ dinv,
                                            const T* __restrict__ xin, T* __restrict__ xout, T* __restrict__ d, T cd,
                                            T cr) {
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    T z = T(0);
#pragma unroll
    for (int s = 0; s < BS; ++s) z += dinv[(a * BS + s) * N + p] * r[s];
    const T dn = (cd != T(0)) ? cd * d[BS * p + a] + cr * z : cr * z;
    d[BS * p + a] = dn;
    xout[BS * p + a] = (xin ? xin[BS * p + a] : T(0)) + dn;
  }
}

template <int BS, int KIND, typename T>
__global__ void __launch_bounds__(256) k_cheb_f(Lat32 L, const T* __restrict__ val, const T* __restrict__ dinv,
                                                const T* __restrict__ b, const T* __restrict__ xin,
                                                T* __restrict__ xout, T* __restrict__ d, T cd, T cr, long long lb) {
  b = lane_ptr(b, lb);
  xin = lane_ptr(xin, lb);
  xout = lane_ptr(xout, lb);
  d = lane_ptr(d, lb);
  const unsigned p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (unsigned)L.N) return;
  T r[BS];
#pragma unroll
  for (int a = 0; a < BS; ++a) r[a] = b[BS * p + a];
  coarse_residual<BS, KIND, f_chunk<BS, T>(), T>(L, p, val, xin, r, 0, 1);
  cheb_update<T, BS>(p, (unsigned)L.N, r, dinv, xin, xout, d, cd, cr);
}

// the first Chebyshev step from x = 0: d = cr D^-1 b, xout = d (no stencil)
template <int BS, typename T>
__global__ void __launch_bounds__(256) k_cheb_zero(long long npts, const T* __restrict__ dinv,
                                                   const T* __restrict__ b, T* __restrict__ xout, T* __restrict__ d,
                                                   T cr, long long lb) {
  b = lane_ptr(b, lb);
  xout = lane_ptr(xout, lb);
  d = lane_ptr(d, lb);
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npts) return;
  T r[BS];
#pragma unroll
  for (int a = 0; a < BS; ++a) r[a] = b[BS * p + a];
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    T z = T(0);
#pragma unroll
    for (int s = 0; s < BS; ++s) z += dinv[(a * BS + s) * npts + p] * r[s];
    d[BS * p + a] = cr * z;
    xout[BS * p + a] = cr * z;
  }
}

// Warp-split offsets: blockDim = (32, W); warp y takes the offsets o with
// o % W == y for 32 consecutive points, so every load instruction reads one
// stored row for 32 consecutive points; the W partial sums meet in shared
// memory and are added in a fixed order.
template <int BS, typename T>
constexpr int w_chunk() { return BS == 6 ? 1 : (sizeof(T) == 4 ? (BS == 1 ? 8 : 2) : (BS == 1 ? 4 : 1)); }

template <int BS, int KIND, int W, typename T>
__device__ __forceinline__ bool wsplit_residual(const Lat32& L, const T* __restrict__ val, const T* __restrict__ x,
                                                T (&part)[W][BS][32], unsigned& p, T r[BS]) {
  p = blockIdx.x * 32 + threadIdx.x;
  const bool valid = p < (unsigned)L.N;
  T acc[BS];
#pragma unroll
  for (int a = 0; a < BS; ++a) acc[a] = T(0);
  if (valid && x) coarse_residual<BS, KIND, w_chunk<BS, T>(), T>(L, p, val, x, acc, threadIdx.y, W);
#pragma unroll
  for (int a = 0; a < BS; ++a) part[threadIdx.y][a][threadIdx.x] = acc[a];
  __syncthreads();
  if (threadIdx.y != 0 || !valid) return false;
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    T s = T(0);
#pragma unroll
    for (int u = 0; u < W; ++u) s += part[u][a][threadIdx.x];
    r[a] = s;  // = -(A x)_a
  }
  return true;
}

template <int BS, int KIND, int W, typename T>
__global__ void __launch_bounds__(32 * W) k_spmv_w(Lat32 L, const T* __restrict__ val, const T* __restrict__ x,
                                                   const T* __restrict__ b, T* __restrict__ y, long long lb) {
  x = lane_ptr(x, lb);
  b = lane_ptr(b, lb);
  y = lane_ptr(y, lb);
  __shared__ T part[W][BS][32];
  unsigned p;
  T r[BS];
  if (!wsplit_residual<BS, KIND, W, T>(L, val, x, part, p, r)) return;
#pragma unroll
  for (int a = 0; a < BS; ++a) y[BS * p + a] = b ? b[BS * p + a] + r[a] : -r[a];
}

template <int BS, int KIND, int W, typename T>
__global__ void __launch_bounds__(32 * W) k_cheb_w(Lat32 L, const T* __restrict__ val, const T* __restrict__ dinv,
                                                   const T* __restrict__ b, const T* __restrict__ xin,
                                                   T* __restrict__ xout, T* __restrict__ d, T cd, T cr, long long lb) {
  b = lane_ptr(b, lb);
  xin = lane_ptr(xin, lb);
  xout = lane_ptr(xout, lb);
  d = lane_ptr(d, lb);
  __shared__ T part[W][BS][32];
  unsigned p;
  T r[BS];
  if (!wsplit_residual<BS, KIND, W, T>(L, val, xin, part, p, r)) return;
#pragma unroll
  for (int a = 0; a < BS; ++a) r[a] += b[BS * p + a];
  cheb_update<T, BS>(p, (unsigned)L.N, r, dinv, xin, xout, d, cd, cr);
}

}  // namespace

template <typename T>
void sweep_spmv(cudaStream_t stream, const StructOp& A, int bs, const T* val, const T* x, const T* b, T* y,
                int sched) {
  const Lat32 L = lat32_of(A);
  dispatch_bs(bs, [&](auto BS) {
    dispatch_kind_bs<BS.value>(A.kind, [&](auto K) {
      dispatch_sched(sched, [&](auto S) {
        if constexpr (S.value == 1)
          k_spmv_f<BS.value, K.value, T><<<lgrid(grid_for(A.N, 256)), 256, 0, stream>>>(L, val, x, b, y, lbytes());
        else
          k_spmv_w<BS.value, K.value, S.value, T><<<lgrid(grid_for(A.N, 32)), dim3(32, S.value), 0, stream>>>(
              L, val, x, b, y, lbytes());
      });
    });
  });
}

template <typename T>
void sweep_cheb(cudaStream_t stream, const StructOp& A, int bs, const T* val, const T* dinv, const T* b,
                const T* xin, T* out, T* d, T cd, T cr, int sched) {
  const Lat32 lat = lat32_of(A);
  dispatch_bs(bs, [&](auto BS) {
    dispatch_kind_bs<BS.value>(A.kind, [&](auto K) {
      dispatch_sched(sched, [&](auto S) {
        if constexpr (S.value == 1)
          k_cheb_f<BS.value, K.value, T><<<lgrid(grid_for(A.N, 256)), 256, 0, stream>>>(lat, val, dinv, b, xin, out, d,
                                                                                         cd, cr, lbytes());
        else
          k_cheb_w<BS.value, K.value, S.value, T><<<lgrid(grid_for(A.N, 32)), dim3(32, S.value), 0, stream>>>(
              lat, val, dinv, b, xin, out, d, cd, cr, lbytes());
      });
    });
  });
}

template <typename T>
void sweep_cheb_zero(cudaStream_t stream, long long npts, int bs, const T* dinv, const T* b, T* out, T* d, T cr) {
  dispatch_bs(bs, [&](auto BS) {
    k_cheb_zero<BS.value, T><<<lgrid(grid_for(npts, 256)), 256, 0, stream>>>(npts, dinv, b, out, d, cr, lbytes());
  });
}

template void sweep_spmv<MHFP_SWEEP_T>(cudaStream_t, const StructOp&, int, const MHFP_SWEEP_T*, const MHFP_SWEEP_T*,
                                       const MHFP_SWEEP_T*, MHFP_SWEEP_T*, int);
template void sweep_cheb<MHFP_SWEEP_T>(cudaStream_t, const StructOp&, int, const MHFP_SWEEP_T*, const MHFP_SWEEP_T*,
                                       const MHFP_SWEEP_T*, const MHFP_SWEEP_T*, MHFP_SWEEP_T*, MHFP_SWEEP_T*,
                                       MHFP_SWEEP_T, MHFP_SWEEP_T, int);
template void sweep_cheb_zero<MHFP_SWEEP_T>(cudaStream_t, long long, int, const MHFP_SWEEP_T*, const MHFP_SWEEP_T*,
                                            MHFP_SWEEP_T*, MHFP_SWEEP_T*, MHFP_SWEEP_T);

}  // namespace mhfp
