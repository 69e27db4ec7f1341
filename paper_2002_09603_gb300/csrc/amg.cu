// Multigrid inner solvers of the block-triangular preconditioner (Section 4,
// Eq. hybridPrec; the paper's M_II^(h) uses smoothed aggregation on A_uu and
// an AMG on C~_pi).  Everything here runs on structured lattices:
//
//  * displacement hierarchy: level 0 = A_uu on the Q1 node lattice (27-point
//    3x3-block stencil); smoothed aggregation with 3x3x3 node aggregates,
//    tentative prolongator = indicator x I_3 on free dofs, one damped block-
//    Jacobi smoothing step of the prolongator, Galerkin coarse operators
//    (which stay 27-point block stencils);
//  * interface-pressure hierarchy: level 0 = C~_pi on faces (11-entry ELL
//    rows), faces -> cells by averaging (weight 1/2 per adjacent cell, 1 on
//    a boundary face, 0 on a drained face) giving a 25-point cell stencil,
//    then scalar smoothed aggregation (125-point coarse stencils);
//  * V(1,1) cycles with Chebyshev smoothing preconditioned by the (block)
//    diagonal, exact dense solve on the last level.
//
// Galerkin products are formed in two deterministic gather passes, Q = A P
// on the fine lattice and A_c = P^T Q per coarse point: no atomics, no
// sparse-matrix hashing.
#include "lattice.cuh"

#include <type_traits>

#include <algorithm>
#include <cmath>

namespace mhfp {

namespace {

// <hot:k_cheb_u0> (bench.py hashes this region to tell whether profiles/traffic.json still applies)
// Chebyshev step: r = b - A xin (r = b when xin is null), d = cd d + cr D^-1 r,
// xout = xin + d.
template <int BS, int KIND, typename T>
__device__ __forceinline__ void cheb_body(const Lat& L, const T* __restrict__ val, const T* __restrict__ dinv,
                                          const T* __restrict__ b, const T* __restrict__ xin, T* __restrict__ xout,
                                          T* __restrict__ d, T cd, T cr) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  T r[BS];
#pragma unroll
  for (int q = 0; q < BS; ++q) r[q] = b[BS * p + q];
  if (xin) {
    int i, j, k;
    L.ijk(p, i, j, k);
#pragma unroll 1
    for (int o = 0; o < St<KIND>::N; ++o) {
      int dx, dy, dz;
      St<KIND>::off(o, dx, dy, dz);
      if (!L.in(i + dx, j + dy, k + dz)) continue;
      const long long q = p + dx + (long long)L.Lx * (dy + (long long)L.Ly * dz);
      const T* v = val + (long long)o * BS * BS * L.N + p;
#pragma unroll
      for (int a = 0; a < BS; ++a)
#pragma unroll
        for (int s = 0; s < BS; ++s) r[a] -= v[(long long)(a * BS + s) * L.N] * xin[BS * q + s];
    }
  }
#pragma unroll
  for (int a = 0; a < BS; ++a) {
    T z = T(0);
#pragma unroll
    for (int s = 0; s < BS; ++s) z += dinv[(long long)(a * BS + s) * L.N + p] * r[s];
    const T dn = (cd != T(0)) ? cd * d[BS * p + a] + cr * z : cr * z;
    d[BS * p + a] = dn;
    xout[BS * p + a] = (xin ? xin[BS * p + a] : T(0)) + dn;
  }
}

template <int BS, int KIND, typename T>
__global__ void __launch_bounds__(256) k_spmv(Lat L, const T* __restrict__ val, const T* __restrict__ x,
                                              const T* __restrict__ b, T* __restrict__ y) {
  spmv_body<BS, KIND, T>(L, val, x, b, y);
}
template <int BS, int KIND, typename T>
__global__ void __launch_bounds__(256) k_cheb(Lat L, const T* __restrict__ val, const T* __restrict__ dinv,
                                              const T* __restrict__ b, const T* __restrict__ xin, T* __restrict__ xout,
                                              T* __restrict__ d, T cd, T cr) {
  cheb_body<BS, KIND, T>(L, val, dinv, b, xin, xout, d, cd, cr);
}
// the finest displacement level (the dominant sweeps) under names of their own
template <typename T>
__global__ void __launch_bounds__(256) k_resid_u0(Lat L, const T* __restrict__ val, const T* __restrict__ x,
                                                  const T* __restrict__ b, T* __restrict__ y, long long lb) {
  spmv_body<3, ST_BOX1, T>(L, val, lane_ptr(x, lb), lane_ptr(b, lb), lane_ptr(y, lb));
}
template <typename T>
__global__ void __launch_bounds__(256) k_cheb_u0(Lat L, const T* __restrict__ val, const T* __restrict__ dinv,
                                                 const T* __restrict__ b, const T* __restrict__ xin,
                                                 T* __restrict__ xout, T* __restrict__ d, T cd, T cr, long long lb) {
  cheb_body<3, ST_BOX1, T>(L, val, dinv, lane_ptr(b, lb), lane_ptr(xin, lb), lane_ptr(xout, lb), lane_ptr(d, lb), cd,
                           cr);
}
// </hot:k_cheb_u0>

// <hot:k_cheb_u0_sym> (hashed like the region above)
// The finest displacement level in FP32 with symmetric storage (A_uu is
// symmetric): per node the diagonal 3x3 block (slot 0) and the blocks
// A(n, n + e_o) of the 13 neighbours with stencil index o = 13 + u > 13
// (slots u = 1..13), i.e. the last 14 offsets of the full layout.  The
// lower blocks are read transposed from the neighbour that owns them:
// A(n, n - e_o) = A(n - e_o, n)^T, slot u of node n - e_o.  Each stored
// block is read by its owner and by one neighbour at most a lattice plane
// apart, so the second read hits L2 and HBM carries each value once.
// Node-blocked layout: nodes in blocks of 32; a block holds its 126 rows
// (slot u, entry e: row 9 u + e) of 32 values each, so the rows a warp
// streams are one contiguous 16 KB range (sym_base).
// UNR slots per loop iteration: 2 keeps two slots' loads in flight (the
// 5-blocks-per-SM variant has the registers for it), 1 one slot.
// lanes of p's warp that hold a node (blocks are whole warps of 32 nodes)
__device__ __forceinline__ unsigned sym_lanes(const Lat& L, long long p) {
  const long long left = L.N - (p & ~31LL);
  return left >= 32 ? 0xffffffffu : ((1u << left) - 1u);
}

// Slot 1 is the +x neighbour, so node p's lower block of that slot is the
// own block of node p - 1, the previous lane's: every lane loads its own
// slot-1 block and the lower one arrives by warp shuffle (lane 0 loads it).
// `mask` holds the lanes of the warp with a node (all lanes call this).
template <typename T, int UNR = 1>
__device__ __forceinline__ void sym_residual(const Lat& L, long long p, const T* __restrict__ up,
                                             const T* __restrict__ x, T r[3], unsigned mask) {
  int i, j, k;
  L.ijk(p, i, j, k);
  const T* own = up + sym_base(p);
  {
    const T x0 = x[3 * p], x1 = x[3 * p + 1], x2 = x[3 * p + 2];
#pragma unroll
    for (int a = 0; a < 3; ++a) r[a] -= own[(3 * a) * 32] * x0 + own[(3 * a + 1) * 32] * x1 + own[(3 * a + 2) * 32] * x2;
  }
  {
    T v[9];
#pragma unroll
    for (int e = 0; e < 9; ++e) v[e] = own[(9 + e) * 32];
    if (i + 1 < L.Lx) {
      const long long q = p + 1;
      const T x0 = x[3 * q], x1 = x[3 * q + 1], x2 = x[3 * q + 2];
#pragma unroll
      for (int a = 0; a < 3; ++a) r[a] -= v[3 * a] * x0 + v[3 * a + 1] * x1 + v[3 * a + 2] * x2;
    }
    const bool first = (threadIdx.x & 31) == 0;
    const T* w = up + sym_base(first && i > 0 ? p - 1 : p) + 9 * 32;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      T t0 = __shfl_up_sync(mask, v[a], 1), t1 = __shfl_up_sync(mask, v[3 + a], 1),
        t2 = __shfl_up_sync(mask, v[6 + a], 1);
      if (first) {
        t0 = w[a * 32];
        t1 = w[(3 + a) * 32];
        t2 = w[(6 + a) * 32];
      }
      if (i > 0) {
        const long long q = p - 1;
        r[a] -= t0 * x[3 * q] + t1 * x[3 * q + 1] + t2 * x[3 * q + 2];
      }
    }
  }
#pragma unroll UNR
  for (int u = 2; u <= 13; ++u) {
    int dx, dy, dz;
    St<ST_BOX1>::off(13 + u, dx, dy, dz);
    const long long s = dx + (long long)L.Lx * (dy + (long long)L.Ly * dz);
    if (L.in(i + dx, j + dy, k + dz)) {
      const long long q = p + s;
      const T* v = own + u * 9 * 32;
      const T x0 = x[3 * q], x1 = x[3 * q + 1], x2 = x[3 * q + 2];
#pragma unroll
      for (int a = 0; a < 3; ++a) r[a] -= v[(3 * a) * 32] * x0 + v[(3 * a + 1) * 32] * x1 + v[(3 * a + 2) * 32] * x2;
    }
    if (L.in(i - dx, j - dy, k - dz)) {
      const long long q = p - s;
      const T* v = up + sym_base(q) + u * 9 * 32;
      const T x0 = x[3 * q], x1 = x[3 * q + 1], x2 = x[3 * q + 2];
#pragma unroll
      for (int a = 0; a < 3; ++a) r[a] -= v[a * 32] * x0 + v[(3 + a) * 32] * x1 + v[(6 + a) * 32] * x2;
    }
  }
}

// MINB resident blocks per SM: 8 (32 registers) fills the SMs in one wave
// when the level has at most 152 x 2048 nodes; 6 (40 registers) keeps more
// loads in flight per thread on larger levels.  The set-up autotuner picks.
template <typename T, int MINB>
__global__ void __launch_bounds__(256, MINB) k_resid_u0_sym(Lat L, const T* __restrict__ up,
                                                            const T* __restrict__ x, const T* __restrict__ b,
                                                            T* __restrict__ y, long long lb) {
  x = lane_ptr(x, lb);
  b = lane_ptr(b, lb);
  y = lane_ptr(y, lb);
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  T r[3] = {b[3 * p], b[3 * p + 1], b[3 * p + 2]};
  sym_residual<T, (MINB <= 5 ? 2 : 1)>(L, p, up, x, r, sym_lanes(L, p));
#pragma unroll
  for (int a = 0; a < 3; ++a) y[3 * p + a] = r[a];
}

template <typename T, int MINB>
__global__ void __launch_bounds__(256, MINB) k_cheb_u0_sym(Lat L, const T* __restrict__ up,
                                                           const T* __restrict__ dinv, const T* __restrict__ b,
                                                           const T* __restrict__ xin, T* __restrict__ xout,
                                                           T* __restrict__ d, T cd, T cr, long long lb) {
  b = lane_ptr(b, lb);
  xin = lane_ptr(xin, lb);
  xout = lane_ptr(xout, lb);
  d = lane_ptr(d, lb);
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  T r[3] = {b[3 * p], b[3 * p + 1], b[3 * p + 2]};
  if (xin) sym_residual<T, (MINB <= 5 ? 2 : 1)>(L, p, up, xin, r, sym_lanes(L, p));
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const T z = dinv[(3 * a) * L.N + p] * r[0] + dinv[(3 * a + 1) * L.N + p] * r[1] + dinv[(3 * a + 2) * L.N + p] * r[2];
    const T dn = (cd != T(0)) ? cd * d[3 * p + a] + cr * z : cr * z;
    d[3 * p + a] = dn;
    xout[3 * p + a] = (xin ? xin[3 * p + a] : T(0)) + dn;
  }
}

// </hot:k_cheb_u0_sym>

// <hot:k_cheb_u0_tma> (hashed like the regions above)
// The same FP32 symmetric-storage sweep and residual, fed by bulk copies.
// A persistent CTA takes node blocks of TMA_NB consecutive nodes.  Its
// producer warp streams, for each block, the 14 stored slots u: the 9 rows
// of the nodes' own blocks A(p, p + e_u) and, for u >= 1, the 9 rows of the
// neighbours' blocks A(p - e_u, p) (read transposed).  In the node-blocked
// layout a slot's 9 rows of one 32-node block are 1152 contiguous bytes, one
// cp.async.bulk copy: 8 for the own rows, 8 or 9 for the transposed ones
// (the node range p - s_u starts anywhere); TMA_S slots in flight; a "full"
// mbarrier per slot buffer counts the bytes, an "empty" one the consumer
// warps that are done with it.  The TMA_NW consumer warps
// (one node per lane) never wait for one another: each waits only for its
// data, and loads the next slot's neighbour x before it waits.  The
// products are summed in the order of sym_residual, so results are
// bit-identical to it.  Every mbarrier wait is bounded: after about 2^31
// clocks the warp records MHFP_WAIT_TIMEOUT in *err and stops; the
// producer waits (bounded) for every copy it issued before the CTA exits.
constexpr int TMA_NW = 8;                    // consumer warps
constexpr int TMA_NB = 32 * TMA_NW;          // nodes per node block
constexpr int TMA_S = 3;                     // slot buffers
constexpr int TMA_CH = 9 * 32;               // floats of one slot of one 32-node block
constexpr int TMA_STAGE = (2 * TMA_NW + 1) * TMA_CH;  // floats per stage: 8 own + 9 transposed chunks
constexpr int TMA_THREADS = 32 * (TMA_NW + 1);
constexpr size_t TMA_SMEM = (size_t)TMA_S * TMA_STAGE * sizeof(float) + 2 * TMA_S * sizeof(unsigned long long);
constexpr int MHFP_WAIT_TIMEOUT = 8;

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
__device__ __forceinline__ void bulk_to_smem(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_addr(dst)),
               "l"(src), "r"(bytes), "r"(smem_addr(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_test(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait for the phase with the given parity; false on timeout
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity) {
  const long long t0 = clock64();
  while (!mbar_test(bar, parity))
    if (clock64() - t0 > (1LL << 31)) return false;
  return true;
}

struct TmaSweep {
  const float* up;   // symmetric half, node-blocked (+ 8 zeroed blocks)
  const float* dinv; // [9][N]
  const float *b, *xin;
  float *xout, *d;
  float cd, cr;
  int* err;
};

// lattice shift of slot u (node p's stored neighbour is p + shift)
__device__ __forceinline__ int sym_shift(const Lat& L, int u) {
  int dx, dy, dz;
  St<ST_BOX1>::off(13 + u, dx, dy, dz);
  return u == 0 ? 0 : dx + L.Lx * (dy + L.Ly * dz);
}

// issue the copies of stage (node block wb, slot u) into buf: own chunks
// 0..7 (the zeroed padding covers the last node block), then the chunks
// holding nodes p0 - s_u .. p0 - s_u + 255, first chunk index clo =
// (p0 - s_u) >> 5; chunks before node 0 are not copied (never read)
__device__ __forceinline__ void tma_issue(const TmaSweep& a, const Lat& L, int wb, int u, float* buf,
                                          unsigned long long* bar) {
  const long long p0 = (long long)wb * TMA_NB;
  const long long c0 = p0 >> 5;
  const unsigned ch_bytes = TMA_CH * 4;
  long long clo = 0;
  int first = 0, last = -1;
  if (u > 0) {
    const long long q0 = p0 - sym_shift(L, u);
    clo = q0 >> 5;
    last = (int)(((q0 + TMA_NB - 1) >> 5) - clo);
    first = clo < 0 ? (int)(-clo) : 0;
  }
  const int ntr = last >= first ? last - first + 1 : 0;
  mbar_expect_tx(bar, (unsigned)(TMA_NW + ntr) * ch_bytes);
#pragma unroll 1
  for (int w = 0; w < TMA_NW; ++w) bulk_to_smem(buf + w * TMA_CH, a.up + ((c0 + w) * 126 + u * 9) * 32, ch_bytes, bar);
#pragma unroll 1
  for (int m = first; m <= last; ++m)
    bulk_to_smem(buf + (TMA_NW + m) * TMA_CH, a.up + ((clo + m) * 126 + u * 9) * 32, ch_bytes, bar);
}

// x of node pc's neighbours in slot u (+s and -s; 0 outside the lattice)
__device__ __forceinline__ void sym_x(const Lat& L, const float* __restrict__ x, long long pc, int i, int j, int k,
                                      int u, float xp[3], float xm[3]) {
  int dx, dy, dz;
  St<ST_BOX1>::off(13 + u, dx, dy, dz);
  const int su = sym_shift(L, u);
  const bool inp = u == 0 || L.in(i + dx, j + dy, k + dz), inm = u > 0 && L.in(i - dx, j - dy, k - dz);
  const long long qp = inp ? pc + su : pc, qm = inm ? pc - su : pc;
#pragma unroll
  for (int e = 0; e < 3; ++e) {
    const float vp = x[3 * qp + e], vm = x[3 * qm + e];
    xp[e] = inp ? vp : 0.f;
    xm[e] = inm ? vm : 0.f;
  }
}

template <bool CHEB>
__global__ void __launch_bounds__(TMA_THREADS, 3) k_sym_tma(Lat L, TmaSweep a0, long long lb) {
  // lane blockIdx.z's vectors (the matrix rows are shared)
  TmaSweep a = a0;
  a.b = lane_ptr(a.b, lb);
  a.xin = lane_ptr(a.xin, lb);
  a.xout = lane_ptr(a.xout, lb);
  a.d = lane_ptr(a.d, lb);
  extern __shared__ __align__(128) unsigned char tma_smem[];
  float* stage = (float*)tma_smem;
  unsigned long long* full = (unsigned long long*)(tma_smem + (size_t)TMA_S * TMA_STAGE * sizeof(float));
  unsigned long long* empty = full + TMA_S;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nblocks = (int)((L.N + TMA_NB - 1) / TMA_NB);
  const int my = (nblocks - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;  // node blocks of this CTA
  const int units = my * 14;
  if (threadIdx.x == 0) {
    for (int s = 0; s < TMA_S; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], TMA_NW);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (warp == TMA_NW) {
    // producer: lane 0 issues every unit once its buffer is free
    if (lane == 0) {
      bool ok = true;
      int g = 0;
      for (; g < units && ok; ++g) {
        const int buf = g % TMA_S;
        if (g >= TMA_S) ok = mbar_wait(&empty[buf], (unsigned)(g / TMA_S - 1) & 1u);
        if (!ok) break;
        tma_issue(a, L, (int)blockIdx.x + (g / 14) * (int)gridDim.x, g % 14, stage + (size_t)buf * TMA_STAGE,
                  &full[buf]);
      }
      // every issued copy lands before the CTA may exit
      for (int h = (g > TMA_S ? g - TMA_S : 0); h < g; ++h)
        if (!mbar_wait(&full[h % TMA_S], (unsigned)(h / TMA_S) & 1u)) ok = false;
      if (!ok) atomicOr(a.err, MHFP_WAIT_TIMEOUT);
    }
  } else {
    bool ok = true;
    int g = 0;
    const int t = warp * 32 + lane;
    for (int k = 0; k < my && ok; ++k) {
      const int wb = (int)blockIdx.x + k * (int)gridDim.x;
      const long long p0 = (long long)wb * TMA_NB;
      const long long p = p0 + t;
      const bool valid = p < L.N;
      const long long pc = valid ? p : L.N - 1;
      int i, j, kk;
      L.ijk(pc, i, j, kk);
      float r[3] = {a.b[3 * pc], a.b[3 * pc + 1], a.b[3 * pc + 2]};
      float xp[3], xm[3];
      sym_x(L, a.xin, pc, i, j, kk, 0, xp, xm);
      for (int u = 0; u < 14; ++u, ++g) {
        const int buf = g % TMA_S;
        // the next slot's x, in flight while this slot's rows are waited for
        float np[3], nm[3];
        sym_x(L, a.xin, pc, i, j, kk, u < 13 ? u + 1 : 13, np, nm);
        // the warp decides together (every lane's wait is bounded)
        if (!__all_sync(0xffffffffu, mbar_wait(&full[buf], (unsigned)(g / TMA_S) & 1u))) {
          ok = false;
          break;
        }
        const float* st = stage + (size_t)buf * TMA_STAGE;
        const float* own = st + warp * TMA_CH + lane;
        if (u == 0) {
#pragma unroll
          for (int e = 0; e < 3; ++e)
            r[e] -= own[(3 * e) * 32] * xp[0] + own[(3 * e + 1) * 32] * xp[1] + own[(3 * e + 2) * 32] * xp[2];
        } else {
          int dx, dy, dz;
          St<ST_BOX1>::off(13 + u, dx, dy, dz);
          if (L.in(i + dx, j + dy, kk + dz)) {
#pragma unroll
            for (int e = 0; e < 3; ++e)
              r[e] -= own[(3 * e) * 32] * xp[0] + own[(3 * e + 1) * 32] * xp[1] + own[(3 * e + 2) * 32] * xp[2];
          }
          if (L.in(i - dx, j - dy, kk - dz)) {
            const long long su = sym_shift(L, u);
            const long long q = p - su;  // >= 0 here
            const int m = (int)((q >> 5) - ((p0 - su) >> 5));
            const float* tr = st + (TMA_NW + m) * TMA_CH + (int)(q & 31);
#pragma unroll
            for (int e = 0; e < 3; ++e)
              r[e] -= tr[e * 32] * xm[0] + tr[(3 + e) * 32] * xm[1] + tr[(6 + e) * 32] * xm[2];
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[buf]);  // this warp is done with the buffer
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          xp[e] = np[e];
          xm[e] = nm[e];
        }
      }
      if (!ok) break;
      if (valid) {
        if (CHEB) {
#pragma unroll
          for (int e = 0; e < 3; ++e) {
            const float z = a.dinv[(3 * e) * L.N + p] * r[0] + a.dinv[(3 * e + 1) * L.N + p] * r[1] +
                            a.dinv[(3 * e + 2) * L.N + p] * r[2];
            const float dn = (a.cd != 0.f) ? a.cd * a.d[3 * p + e] + a.cr * z : a.cr * z;
            a.d[3 * p + e] = dn;
            a.xout[3 * p + e] = a.xin[3 * p + e] + dn;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 3; ++e) a.xout[3 * p + e] = r[e];
        }
      }
    }
    if (!ok && lane == 0) atomicOr(a.err, MHFP_WAIT_TIMEOUT);
  }
  __syncthreads();  // no warp leaves while copies into this CTA's shared memory may be in flight
}
// </hot:k_cheb_u0_tma>

// ---------------------------------------------------------------- transfers
// Prolongation x += P x_c and restriction b_c = P^T r between lattice levels,
// with the same 32-bit indexing and batched loads as the sweeps.  P is
// stored [ns^3 slots][BF x BC][fine points] (BF unknowns per fine point, BC
// per coarse point: 3 x 3 or 1 x 1 for M_II^(h), 3 x 6 and 6 x 6 with the
// rigid-body modes); slot (sx, sy, sz) of fine point (a, b, c) is coarse
// point (p_lo(a) + sx, p_lo(b) + sy, p_lo(c) + sz).  An absent coarse point
// contributes 0 (a select, not a multiply).
template <int BF, int BC, int R, int CH, typename T>
__device__ __forceinline__ void prolong_sum(const Lat32& F, const Lat32& C, unsigned p, const T* __restrict__ P,
                                            const T* __restrict__ xc, T acc[BF], int first, int step) {
  constexpr int ns = (2 + 2 * R) / 3 + 1, NS = ns * ns * ns;
  int a, b, c;
  F.ijk(p, a, b, c);
  const int lx = p_lo(a, R), ly = p_lo(b, R), lz = p_lo(c, R);
  bool vx[ns], vy[ns], vz[ns];
#pragma unroll
  for (int t = 0; t < ns; ++t) {
    vx[t] = (unsigned)(lx + t) < (unsigned)C.Lx;
    vy[t] = (unsigned)(ly + t) < (unsigned)C.Ly;
    vz[t] = (unsigned)(lz + t) < (unsigned)C.Lz;
  }
  const unsigned N = (unsigned)F.N;
#pragma unroll
  for (int s0 = 0; s0 < NS; s0 += CH) {
    T pv[CH][BF * BC], xv[CH][BC];
#pragma unroll
    for (int q = 0; q < CH; ++q) {
      const int sl = s0 + q;
      if (sl < NS && sl % step == first) {
        const int sx = sl % ns, sy = (sl / ns) % ns, sz = sl / (ns * ns);
        const bool in = vx[sx] && vy[sy] && vz[sz];
        const unsigned J = in ? (unsigned)(lx + sx) + (unsigned)C.Lx * ((unsigned)(ly + sy) + (unsigned)C.Ly * (unsigned)(lz + sz)) : 0u;
#pragma unroll
        for (int e = 0; e < BF * BC; ++e) {
          const T v = P[(unsigned)(sl * BF * BC + e) * N + p];
          pv[q][e] = in ? v : T(0);
        }
#pragma unroll
        for (int t = 0; t < BC; ++t) {
          const T v = xc[BC * J + t];
          xv[q][t] = in ? v : T(0);
        }
      }
    }
#pragma unroll
    for (int q = 0; q < CH; ++q)
      if (s0 + q < NS && (s0 + q) % step == first)
#pragma unroll
        for (int r = 0; r < BF; ++r)
#pragma unroll
          for (int t = 0; t < BC; ++t) acc[r] += pv[q][r * BC + t] * xv[q][t];
  }
}

template <int BF, int BC>
constexpr int prolong_chunk() { return BF * BC == 1 ? 9 : (BF * BC <= 9 ? 4 : 1); }

// one fine point per thread
template <int BF, int BC, int R, typename T>
__global__ void __launch_bounds__(256) k_prolong_f(Lat32 F, Lat32 C, const T* __restrict__ P,
                                                   const T* __restrict__ xc, T* __restrict__ x, long long lb) {
  xc = lane_ptr(xc, lb);
  x = lane_ptr(x, lb);
  // blocks take the fine points in descending order: the restriction just
  // streamed P in ascending order, so its tail is still in L2
  const unsigned p = (gridDim.x - 1 - blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= (unsigned)F.N) return;
  T acc[BF];
#pragma unroll
  for (int r = 0; r < BF; ++r) acc[r] = T(0);
  prolong_sum<BF, BC, R, prolong_chunk<BF, BC>(), T>(F, C, p, P, xc, acc, 0, 1);
#pragma unroll
  for (int r = 0; r < BF; ++r) x[BF * p + r] += acc[r];
}

// small fine levels: the slots split over W warps for 32 consecutive fine
// points, partial sums added in a fixed order through shared memory
template <int BF, int BC, int R, int W, typename T>
__global__ void __launch_bounds__(32 * W) k_prolong_w(Lat32 F, Lat32 C, const T* __restrict__ P,
                                                      const T* __restrict__ xc, T* __restrict__ x, long long lb) {
  xc = lane_ptr(xc, lb);
  x = lane_ptr(x, lb);
  __shared__ T part[W][BF][32];
  const unsigned p = blockIdx.x * 32 + threadIdx.x;
  const bool valid = p < (unsigned)F.N;
  T acc[BF];
#pragma unroll
  for (int r = 0; r < BF; ++r) acc[r] = T(0);
  if (valid) prolong_sum<BF, BC, R, (BF * BC > 9 ? 1 : 2), T>(F, C, p, P, xc, acc, threadIdx.y, W);
#pragma unroll
  for (int r = 0; r < BF; ++r) part[threadIdx.y][r][threadIdx.x] = acc[r];
  __syncthreads();
  if (threadIdx.y != 0 || !valid) return;
#pragma unroll
  for (int r = 0; r < BF; ++r) {
    T sum = T(0);
#pragma unroll
    for (int u = 0; u < W; ++u) sum += part[u][r][threadIdx.x];
    x[BF * p + r] += sum;
  }
}

// restriction b_c = P^T r, one warp per coarse point: the lanes split the
// (3 + 2R)^3 fine box around it, each lane issuing the loads of all its box
// points before the sums, then a fixed-order xor reduction over the warp
template <int BF, int BC, int R, typename T>
__global__ void __launch_bounds__(256) k_restrict_f(Lat32 F, Lat32 C, const T* __restrict__ P,
                                                    const T* __restrict__ r, T* __restrict__ bc,
                                                    const T* __restrict__ dinvc, T cr, T* __restrict__ xc,
                                                    T* __restrict__ dc, long long lb) {
  r = lane_ptr(r, lb);
  bc = lane_ptr(bc, lb);
  xc = lane_ptr(xc, lb);
  dc = lane_ptr(dc, lb);
  constexpr int ns = (2 + 2 * R) / 3 + 1, w = 3 + 2 * R, NB = w * w * w, PER = (NB + 31) / 32;
  // blocks larger than 3 x 3 keep one box point's loads in flight at a time
  constexpr int KB = BF * BC > 9 ? 1 : PER;
  const unsigned J = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  const bool valid = J < (unsigned)C.N;
  T acc[BC];
#pragma unroll
  for (int q = 0; q < BC; ++q) acc[q] = T(0);
  if (valid) {
    int I, Jj, K;
    C.ijk(J, I, Jj, K);
    const unsigned N = (unsigned)F.N;
#pragma unroll
    for (int k0 = 0; k0 < PER; k0 += KB) {
      T pv[KB][BF * BC], rv[KB][BF];
#pragma unroll
      for (int kk = 0; kk < KB; ++kk) {
        const int e = lane + 32 * (k0 + kk);
        const int ex = e % w, ey = (e / w) % w, ez = e / (w * w);
        const int a = 3 * I - R + ex, b = 3 * Jj - R + ey, c = 3 * K - R + ez;
        const bool in = e < NB && (unsigned)a < (unsigned)F.Lx && (unsigned)b < (unsigned)F.Ly &&
                        (unsigned)c < (unsigned)F.Lz;
        const int sx = I - p_lo(a, R), sy = Jj - p_lo(b, R), sz = K - p_lo(c, R);
        const bool ok = in && (unsigned)sx < (unsigned)ns && (unsigned)sy < (unsigned)ns && (unsigned)sz < (unsigned)ns;
        const unsigned fp = ok ? (unsigned)a + (unsigned)F.Lx * ((unsigned)b + (unsigned)F.Ly * (unsigned)c) : 0u;
        const int sl = ok ? sx + ns * (sy + ns * sz) : 0;
#pragma unroll
        for (int t = 0; t < BF * BC; ++t) {
          const T v = P[(unsigned)(sl * BF * BC + t) * N + fp];
          pv[kk][t] = ok ? v : T(0);
        }
#pragma unroll
        for (int t = 0; t < BF; ++t) {
          const T v = r[BF * fp + t];
          rv[kk][t] = ok ? v : T(0);
        }
      }
#pragma unroll
      for (int kk = 0; kk < KB; ++kk)
#pragma unroll
        for (int q = 0; q < BC; ++q)
#pragma unroll
          for (int t = 0; t < BF; ++t) acc[q] += pv[kk][t * BC + q] * rv[kk][t];
    }
  }
#pragma unroll
  for (int q = 0; q < BC; ++q) {
#pragma unroll
    for (int m = 16; m > 0; m >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], m);
    if (valid && lane == 0) bc[BC * J + q] = acc[q];
  }
  // the coarse level's first Chebyshev step from zero (with dinvc): d = cr
  // D^-1 b, x = d, the same sums as its own kernel would form from bc
  if (dinvc && valid && lane == 0) {
    const unsigned Nc = (unsigned)C.N;
#pragma unroll
    for (int a = 0; a < BC; ++a) {
      T z = T(0);
#pragma unroll
      for (int t = 0; t < BC; ++t) z += dinvc[(unsigned)(a * BC + t) * Nc + J] * acc[t];
      dc[BC * J + a] = cr * z;
      xc[BC * J + a] = cr * z;
    }
  }
}

// face level (ELL, 11 slots) versions
// y = b - C x (y = C x when b is null) on the face level; the 11 columns of
// each row follow from the face topology (FaceTopo32::ell_cols), so only
// the values stream from memory
template <typename T>
__global__ void __launch_bounds__(256) k_spmv_ell(FaceTopo32 t, const T* __restrict__ val, const T* __restrict__ x,
                                                  const T* __restrict__ b, T* __restrict__ y, long long lb) {
  x = lane_ptr(x, lb);
  b = lane_ptr(b, lb);
  y = lane_ptr(y, lb);
  const unsigned f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= t.nF) return;
  unsigned col[11];
  t.ell_cols(f, col);
  T a = T(0);
#pragma unroll
  for (int q = 0; q < 11; ++q) a += val[q * t.nF + f] * x[col[q]];
  y[f] = b ? b[f] - a : a;
}

template <typename T>
__global__ void __launch_bounds__(256) k_cheb_ell(FaceTopo32 t, const T* __restrict__ val,
                                                  const T* __restrict__ dinv, const T* __restrict__ b,
                                                  const T* __restrict__ xin, T* __restrict__ xout, T* __restrict__ d,
                                                  T cd, T cr, long long lb) {
  b = lane_ptr(b, lb);
  xin = lane_ptr(xin, lb);
  xout = lane_ptr(xout, lb);
  d = lane_ptr(d, lb);
  const unsigned f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= t.nF) return;
  T r = b[f];
  if (xin) {
    unsigned col[11];
    t.ell_cols(f, col);
#pragma unroll
    for (int q = 0; q < 11; ++q) r -= val[q * t.nF + f] * xin[col[q]];
  }
  const T dn = (cd != T(0)) ? cd * d[f] + cr * dinv[f] * r : cr * dinv[f] * r;
  d[f] = dn;
  xout[f] = (xin ? xin[f] : T(0)) + dn;
}

// faces -> cells Galerkin product of the interface-pressure hierarchy (set-up)
struct FaceTopo {
  int nx, ny, nz;
  long long nT, nF, nFx, nFy;
};

__device__ __forceinline__ long long ft_cell_face(const FaceTopo& d, int i, int j, int k, int lf) {
  switch (lf) {
    case 0: return i + (long long)(d.nx + 1) * (j + (long long)d.ny * k);
    case 1: return (i + 1) + (long long)(d.nx + 1) * (j + (long long)d.ny * k);
    case 2: return d.nFx + i + (long long)d.nx * (j + (long long)(d.ny + 1) * k);
    case 3: return d.nFx + i + (long long)d.nx * ((j + 1) + (long long)(d.ny + 1) * k);
    case 4: return d.nFx + d.nFy + i + (long long)d.nx * (j + (long long)d.ny * k);
    default: return d.nFx + d.nFy + i + (long long)d.nx * (j + (long long)d.ny * (k + 1));
  }
}

// face -> up to two cells as lattice coordinates (valid flags)
__device__ __forceinline__ int ft_face_cells(const FaceTopo& d, long long f, int c[2][3]) {
  int i, j, k, ax;
  if (f < d.nFx) {
    ax = 0; i = (int)(f % (d.nx + 1)); long long r = f / (d.nx + 1); j = (int)(r % d.ny); k = (int)(r / d.ny);
  } else if (f < d.nFx + d.nFy) {
    long long g = f - d.nFx;
    ax = 1; i = (int)(g % d.nx); long long r = g / d.nx; j = (int)(r % (d.ny + 1)); k = (int)(r / (d.ny + 1));
  } else {
    long long g = f - d.nFx - d.nFy;
    ax = 2; i = (int)(g % d.nx); long long r = g / d.nx; j = (int)(r % d.ny); k = (int)(r / d.ny);
  }
  const int lim[3] = {d.nx, d.ny, d.nz};
  int cnt = 0;
  int base[3] = {i, j, k};
  base[ax] -= 1;
  if (base[ax] >= 0) { c[cnt][0] = base[0]; c[cnt][1] = base[1]; c[cnt][2] = base[2]; ++cnt; }
  base[ax] += 1;
  if (base[ax] < lim[ax]) { c[cnt][0] = base[0]; c[cnt][1] = base[1]; c[cnt][2] = base[2]; ++cnt; }
  return cnt;
}

template <typename T>
__global__ void __launch_bounds__(256) k_restrict_faces(FaceTopo32 t, const T* __restrict__ pw,
                                                        const T* __restrict__ r, T* __restrict__ bc,
                                                        const T* __restrict__ dinvc, T cr, T* __restrict__ xc,
                                                        T* __restrict__ dc, long long lb) {
  r = lane_ptr(r, lb);
  bc = lane_ptr(bc, lb);
  xc = lane_ptr(xc, lb);
  dc = lane_ptr(dc, lb);
  const unsigned Tc = blockIdx.x * blockDim.x + threadIdx.x;
  if (Tc >= t.nT) return;
  const unsigned q = t.d_nx.div(Tc);
  const int i = (int)(Tc - q * (unsigned)t.nx);
  const int k = (int)t.d_ny.div(q), j = (int)(q - (unsigned)k * (unsigned)t.ny);
  T s = T(0);
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) {
    const unsigned f = t.face(i, j, k, lf);
    s += pw[f] * r[f];
  }
  bc[Tc] = s;
  if (dinvc) {  // the cell level's first Chebyshev step from zero, as k_restrict_f
    T z = T(0);
    z += dinvc[Tc] * s;
    dc[Tc] = cr * z;
    xc[Tc] = cr * z;
  }
}

template <typename T>
__global__ void __launch_bounds__(256) k_prolong_faces(FaceTopo32 t, const T* __restrict__ pw,
                                                       const T* __restrict__ xc, T* __restrict__ x, long long lb) {
  xc = lane_ptr(xc, lb);
  x = lane_ptr(x, lb);
  // descending block order, as k_prolong_f
  const unsigned f = (gridDim.x - 1 - blockIdx.x) * blockDim.x + threadIdx.x;
  if (f >= t.nF) return;
  int c[2][3], lf[2];
  bool ok[2];
  t.cells(f, c, ok, lf);
  T s = T(0);
#pragma unroll
  for (int q = 0; q < 2; ++q)
    if (ok[q]) s += xc[t.cell(c[q][0], c[q][1], c[q][2])];
  x[f] += pw[f] * s;
}

// dense coarsest solve y = Ainv b, one block of 256 threads per row (each
// thread a strided slice of the row, then a fixed-order block sum); the
// inverse and the sums stay FP64 whatever the precision of the cycle's vectors
template <typename T>
__global__ void __launch_bounds__(256) k_dense_mv(int n, const double* __restrict__ Ainv, const T* __restrict__ b,
                                                  T* __restrict__ y, long long lb) {
  b = lane_ptr(b, lb);
  y = lane_ptr(y, lb);
  // y = Ainv b (the coarsest level's dense FP64 inverse): a block of 8 warps
  // takes 2 rows, each row's columns split in quarters, one warp per
  // quarter, so that about 40 warps per SM keep the inverse streaming; the
  // four partial sums of a row are added in a fixed order
  __shared__ double part[8];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int row = blockIdx.x * 2 + (warp >> 2);
  const int chunk = (n + 3) / 4;
  const int c0 = (warp & 3) * chunk, c1 = min(n, c0 + chunk);
  double s = 0.0;
  if (row < n) {
    const double* a = Ainv + (long long)row * n;
#pragma unroll 4
    for (int c = c0 + lane; c < c1; c += 32) s += a[c] * (double)b[c];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) part[warp] = s;
  __syncthreads();
  if (threadIdx.x < 2) {
    const int r = blockIdx.x * 2 + threadIdx.x;
    if (r < n) y[r] = (T)(((part[4 * threadIdx.x] + part[4 * threadIdx.x + 1]) + part[4 * threadIdx.x + 2]) +
                          part[4 * threadIdx.x + 3]);
  }
}

__global__ void k_cast_f32(long long n, const double* __restrict__ x, float* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

// rows 0..125 of the FP64 offset-major values ([row][n]) into the
// node-blocked FP32 layout of the symmetric sweep
__global__ void k_cast_f32_sym(long long n, const double* __restrict__ x, float* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 126 * n) return;
  const long long row = i / n, q = i % n;
  y[sym_base(q) + 32 * row] = (float)x[i];
}

// ------------------------------------------------------------------ setup
template <int BS, int KIND>
__global__ void k_dinv(Lat L, const double* __restrict__ val, double* __restrict__ dinv) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= L.N) return;
  const double* v = val + (long long)St<KIND>::C * BS * BS * L.N + p;
  if (BS == 1) {
    dinv[p] = 1.0 / v[0];
  } else if (BS != 3) {
    // the SPD point block of the rigid-body-mode levels (6 x 6): Gauss-
    // Jordan elimination without pivoting (positive pivots of an SPD block)
    double m[BS][2 * BS];
    for (int r = 0; r < BS; ++r)
      for (int c = 0; c < BS; ++c) {
        m[r][c] = v[(long long)(r * BS + c) * L.N];
        m[r][BS + c] = (r == c) ? 1.0 : 0.0;
      }
    for (int c = 0; c < BS; ++c) {
      const double ip = 1.0 / m[c][c];
      for (int k = 0; k < 2 * BS; ++k) m[c][k] *= ip;
      for (int r = 0; r < BS; ++r) {
        if (r == c) continue;
        const double f = m[r][c];
        for (int k = 0; k < 2 * BS; ++k) m[r][k] -= f * m[c][k];
      }
    }
    for (int r = 0; r < BS; ++r)
      for (int c = 0; c < BS; ++c) dinv[(long long)(r * BS + c) * L.N + p] = m[r][BS + c];
  } else {
    double a[9];
    for (int q = 0; q < 9; ++q) a[q] = v[(long long)q * L.N];
    const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
    const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
    const double id = 1.0 / det;
    double inv[9];
    inv[0] = c00 * id; inv[1] = (a[2] * a[7] - a[1] * a[8]) * id; inv[2] = (a[1] * a[5] - a[2] * a[4]) * id;
    inv[3] = c01 * id; inv[4] = (a[0] * a[8] - a[2] * a[6]) * id; inv[5] = (a[2] * a[3] - a[0] * a[5]) * id;
    inv[6] = c02 * id; inv[7] = (a[1] * a[6] - a[0] * a[7]) * id; inv[8] = (a[0] * a[4] - a[1] * a[3]) * id;
    for (int q = 0; q < 9; ++q) dinv[(long long)q * L.N + p] = inv[q];
  }
}

__global__ void k_dinv_ell(long long n, const double* __restrict__ val, double* __restrict__ dinv) {
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f < n) dinv[f] = 1.0 / val[f];
}

// y = D^-1 x (block), x and y of length BS*N
template <int BS>
__global__ void k_apply_dinv(long long N, const double* __restrict__ dinv, const double* __restrict__ x,
                             double* __restrict__ y) {
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  for (int a = 0; a < BS; ++a) {
    double s = 0.0;
    for (int t = 0; t < BS; ++t) s += dinv[(long long)(a * BS + t) * N + p] * x[BS * p + t];
    y[BS * p + a] = s;
  }
}

__global__ void k_power_start(long long n, double* __restrict__ v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = 1.0 + (double)((7919LL * i) % 97) / 97.0;
}

__global__ void k_scale_by(long long n, double s, double* __restrict__ v) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] *= s;
}

// Smoothed prolongator: P[a, J] = [a in J] diag(active_a) - omega D_a^-1 sum_{b in J, b ~ a} A_ab diag(active_b)
template <int BS, int KIND>
__global__ void k_build_P(Lat F, Lat Cc, const double* __restrict__ val, const double* __restrict__ dinv,
                          const unsigned char* __restrict__ active, double omega, double* __restrict__ P) {
  const int R = St<KIND>::R;
  const int ns = p_slots(R);
  const int nslot = ns * ns * ns;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= F.N * nslot) return;
  const int s = (int)(tid / F.N);
  const long long p = tid - (long long)s * F.N;
  int a, b, c;
  F.ijk(p, a, b, c);
  const int sx = s % ns, sy = (s / ns) % ns, sz = s / (ns * ns);
  const int I = p_lo(a, R) + sx, J = p_lo(b, R) + sy, K = p_lo(c, R) + sz;
  double out[BS * BS];
  for (int q = 0; q < BS * BS; ++q) out[q] = 0.0;
  if (Cc.in(I, J, K)) {
    double ap[BS * BS];
    for (int q = 0; q < BS * BS; ++q) ap[q] = 0.0;
    for (int o = 0; o < St<KIND>::N; ++o) {
      int dx, dy, dz;
      St<KIND>::off(o, dx, dy, dz);
      const int na = a + dx, nb = b + dy, nc = c + dz;
      if (!F.in(na, nb, nc)) continue;
      if (na / 3 != I || nb / 3 != J || nc / 3 != K) continue;
      const long long q = F.id(na, nb, nc);
      const double* v = val + (long long)o * BS * BS * F.N + p;
      for (int r = 0; r < BS; ++r)
        for (int t = 0; t < BS; ++t) ap[r * BS + t] += v[(long long)(r * BS + t) * F.N] * (active[BS * q + t] ? 1.0 : 0.0);
    }
    for (int r = 0; r < BS; ++r)
      for (int t = 0; t < BS; ++t) {
        double z = 0.0;
        for (int u = 0; u < BS; ++u) z += dinv[(long long)(r * BS + u) * F.N + p] * ap[u * BS + t];
        out[r * BS + t] = -omega * z;
      }
    if (a / 3 == I && b / 3 == J && c / 3 == K)
      for (int r = 0; r < BS; ++r) out[r * BS + r] += active[BS * p + r] ? 1.0 : 0.0;
  }
  for (int q = 0; q < BS * BS; ++q) P[((long long)s * BS * BS + q) * F.N + p] = out[q];
}

template <int BS>
__global__ void k_active_coarse(Lat F, Lat Cc, const unsigned char* __restrict__ af, unsigned char* __restrict__ ac) {
  const long long J = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (J >= Cc.N) return;
  int I, Jj, K;
  Cc.ijk(J, I, Jj, K);
  unsigned char m[BS];
  for (int q = 0; q < BS; ++q) m[q] = 0;
  for (int c = 3 * K; c < 3 * K + 3 && c < F.Lz; ++c)
    for (int b = 3 * Jj; b < 3 * Jj + 3 && b < F.Ly; ++b)
      for (int a = 3 * I; a < 3 * I + 3 && a < F.Lx; ++a) {
        const long long p = F.id(a, b, c);
        for (int q = 0; q < BS; ++q) m[q] |= af[BS * p + q];
      }
  for (int q = 0; q < BS; ++q) ac[BS * J + q] = m[q] ? 1 : 0;
}

// Q[a, J] = sum_o A[a, a+o] P[a+o, J]   (fine point a, coarse J in its Q range;
// A blocks BF x BF, P and Q blocks BF x BC)
template <int BF, int BC, int KIND>
__global__ void k_build_Q(Lat F, Lat Cc, const double* __restrict__ val, const double* __restrict__ P,
                          double* __restrict__ Q) {
  const int R = St<KIND>::R;
  const int ns = p_slots(R), nq = q_slots(R);
  const int nqs = nq * nq * nq;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= F.N * nqs) return;
  const int s = (int)(tid / F.N);
  const long long p = tid - (long long)s * F.N;
  int a, b, c;
  F.ijk(p, a, b, c);
  const int I = q_lo(a, R) + s % nq, J = q_lo(b, R) + (s / nq) % nq, K = q_lo(c, R) + s / (nq * nq);
  double out[BF * BC];
  for (int q = 0; q < BF * BC; ++q) out[q] = 0.0;
  if (Cc.in(I, J, K)) {
    for (int o = 0; o < St<KIND>::N; ++o) {
      int dx, dy, dz;
      St<KIND>::off(o, dx, dy, dz);
      const int na = a + dx, nb = b + dy, nc = c + dz;
      if (!F.in(na, nb, nc)) continue;
      const int px = I - p_lo(na, R), py = J - p_lo(nb, R), pz = K - p_lo(nc, R);
      if (px < 0 || px >= ns || py < 0 || py >= ns || pz < 0 || pz >= ns) continue;
      const long long q = F.id(na, nb, nc);
      const int ps = px + ns * (py + ns * pz);
      const double* v = val + (long long)o * BF * BF * F.N + p;
      const double* pv = P + (long long)ps * BF * BC * F.N + q;
      for (int r = 0; r < BF; ++r)
        for (int t = 0; t < BC; ++t) {
          double z = 0.0;
          for (int u = 0; u < BF; ++u) z += v[(long long)(r * BF + u) * F.N] * pv[(long long)(u * BC + t) * F.N];
          out[r * BC + t] += z;
        }
    }
  }
  for (int q = 0; q < BF * BC; ++q) Q[((long long)s * BF * BC + q) * F.N + p] = out[q];
}

// A_c[J, J+oc] = sum_{a in box(J)} P[a, J]^T Q[a, J+oc]   (BC x BC blocks)
template <int BF, int BC, int CKIND>
__global__ void k_rap(Lat F, Lat Cc, int R, const double* __restrict__ P, const double* __restrict__ Q,
                      const unsigned char* __restrict__ ac, double* __restrict__ Ac) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= Cc.N * St<CKIND>::N) return;
  const int oc = (int)(tid / Cc.N);
  const long long J = tid - (long long)oc * Cc.N;
  int I, Jj, K;
  Cc.ijk(J, I, Jj, K);
  int ox, oy, oz;
  St<CKIND>::off(oc, ox, oy, oz);
  const int I2 = I + ox, J2 = Jj + oy, K2 = K + oz;
  double out[BC * BC];
  for (int q = 0; q < BC * BC; ++q) out[q] = 0.0;
  if (Cc.in(I2, J2, K2)) {
    const int ns = p_slots(R), nq = q_slots(R);
    for (int c = 3 * K - R; c <= 3 * K + 2 + R; ++c) {
      if (c < 0 || c >= F.Lz) continue;
      const int pz = K - p_lo(c, R), qz = K2 - q_lo(c, R);
      if (pz < 0 || pz >= ns || qz < 0 || qz >= nq) continue;
      for (int b = 3 * Jj - R; b <= 3 * Jj + 2 + R; ++b) {
        if (b < 0 || b >= F.Ly) continue;
        const int py = Jj - p_lo(b, R), qy = J2 - q_lo(b, R);
        if (py < 0 || py >= ns || qy < 0 || qy >= nq) continue;
        for (int a = 3 * I - R; a <= 3 * I + 2 + R; ++a) {
          if (a < 0 || a >= F.Lx) continue;
          const int px = I - p_lo(a, R), qx = I2 - q_lo(a, R);
          if (px < 0 || px >= ns || qx < 0 || qx >= nq) continue;
          const long long p = F.id(a, b, c);
          const double* pv = P + (long long)(px + ns * (py + ns * pz)) * BF * BC * F.N + p;
          const double* qv = Q + (long long)(qx + nq * (qy + nq * qz)) * BF * BC * F.N + p;
          for (int r = 0; r < BC; ++r)
            for (int t = 0; t < BC; ++t) {
              double z = 0.0;
              for (int u = 0; u < BF; ++u) z += pv[(long long)(u * BC + r) * F.N] * qv[(long long)(u * BC + t) * F.N];
              out[r * BC + t] += z;
            }
        }
      }
    }
  }
  if (ox == 0 && oy == 0 && oz == 0)
    for (int r = 0; r < BC; ++r)
      if (!ac[BC * J + r]) out[r * BC + r] = 1.0;
  for (int q = 0; q < BC * BC; ++q) Ac[((long long)oc * BC * BC + q) * Cc.N + J] = out[q];
}

// ------------------------------------------- rigid-body-mode near-kernel
// M_III^(h) (Section 5: smoothed aggregation with the six rigid-body modes
// as the near-kernel of A_uu).  Per aggregate (3x3x3 box of lattice points)
// one warp factorises the near-kernel restricted to the aggregate's dofs,
// N_K = Q_K R_K, by classical Gram-Schmidt applied twice in mode order
// (translations x, y, z, rotations about x, y, z); a mode left with at
// most 1e-10 of its norm is dropped (zero column of Q_K, zero row of R_K,
// the coarse dof inactive).  The lanes hold the rows (lane l: rows l,
// l + 32, ...), dot products are fixed-order xor butterflies.  Q_K is
// stored per fine point, Pt[(a BC + j)][p] = Q_K(row of dof a of point p, j);
// R_K as the coarse point's near-kernel, Nc[(a 6 + j)][K] = R_K(a, j).
constexpr int RBM_K = 6;
constexpr double RBM_DROP = 1e-10;

__device__ __forceinline__ double warp_sum_xor(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += __shfl_xor_sync(0xffffffffu, v, m);
  return v;
}

// near-kernel rows of the aggregate's dofs: the fine level (BF = 3) takes
// the rigid-body modes of the node coordinates (about the centroid cen,
// rows of prescribed dofs zero); a coarse level (BF = 6) takes the previous
// level's R blocks
template <int BF>
__device__ __forceinline__ void rbm_rows(const Lat& F, int I, int J, int K, int row, const double* __restrict__ coords,
                                         const unsigned char* __restrict__ active, const double* __restrict__ Nprev,
                                         double cx, double cy, double cz, double n[RBM_K], long long& p, int& a,
                                         bool& ok) {
  // row = local point (box order, i fastest) * BF + dof
  const int lp = row / BF;
  a = row - lp * BF;
  const int ex = lp % 3, ey = (lp / 3) % 3, ez = lp / 9;
  const int i = 3 * I + ex, j = 3 * J + ey, k = 3 * K + ez;
  ok = lp < 27 && F.in(i, j, k);
  p = ok ? F.id(i, j, k) : 0;
  for (int m = 0; m < RBM_K; ++m) n[m] = 0.0;
  if (!ok || !active[BF * p + a]) return;
  if (BF == 3) {
    const double x = coords[3 * p] - cx, y = coords[3 * p + 1] - cy, z = coords[3 * p + 2] - cz;
    n[a] = 1.0;
    // rotation about x: (0, -z, y); about y: (z, 0, -x); about z: (-y, x, 0)
    if (a == 0) { n[4] = z; n[5] = -y; }
    if (a == 1) { n[3] = -z; n[5] = x; }
    if (a == 2) { n[3] = y; n[4] = -x; }
  } else {
    for (int m = 0; m < RBM_K; ++m) n[m] = Nprev[(long long)(a * RBM_K + m) * F.N + p];
  }
}

template <int BF, int RPL>
__global__ void __launch_bounds__(128) k_rbm_tentative(Lat F, Lat Cc, const double* __restrict__ coords,
                                                        const unsigned char* __restrict__ active,
                                                        const double* __restrict__ Nprev, double cx, double cy,
                                                        double cz, double* __restrict__ Pt, double* __restrict__ Nc,
                                                        unsigned char* __restrict__ ac) {
  const long long Kc = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (Kc >= Cc.N) return;  // whole warps leave together
  int I, J, K;
  Cc.ijk(Kc, I, J, K);
  double v[RPL][RBM_K], q[RPL][RBM_K];
  long long pp[RPL];
  int aa[RPL];
  bool ok[RPL];
#pragma unroll
  for (int t = 0; t < RPL; ++t) {
    rbm_rows<BF>(F, I, J, K, lane + 32 * t, coords, active, Nprev, cx, cy, cz, v[t], pp[t], aa[t], ok[t]);
#pragma unroll
    for (int m = 0; m < RBM_K; ++m) q[t][m] = 0.0;
  }
  double R[RBM_K][RBM_K];
#pragma unroll
  for (int a = 0; a < RBM_K; ++a)
#pragma unroll
    for (int b = 0; b < RBM_K; ++b) R[a][b] = 0.0;
  bool kept[RBM_K];
#pragma unroll
  for (int j = 0; j < RBM_K; ++j) {
    double w[RPL];
    double s0 = 0.0;
#pragma unroll
    for (int t = 0; t < RPL; ++t) {
      w[t] = v[t][j];
      s0 += w[t] * w[t];
    }
    const double n0 = sqrt(warp_sum_xor(s0));
#pragma unroll
    for (int pass = 0; pass < 2; ++pass) {
      double h[RBM_K];
#pragma unroll
      for (int i = 0; i < RBM_K; ++i) {
        if (i >= j) break;
        double d = 0.0;
#pragma unroll
        for (int t = 0; t < RPL; ++t) d += q[t][i] * w[t];
        h[i] = warp_sum_xor(d);
      }
#pragma unroll
      for (int i = 0; i < RBM_K; ++i) {
        if (i >= j) break;
        R[i][j] += h[i];
#pragma unroll
        for (int t = 0; t < RPL; ++t) w[t] -= h[i] * q[t][i];
      }
    }
    double s1 = 0.0;
#pragma unroll
    for (int t = 0; t < RPL; ++t) s1 += w[t] * w[t];
    const double nv = sqrt(warp_sum_xor(s1));
    kept[j] = n0 > 0.0 && nv > RBM_DROP * n0;
    const double inv = kept[j] ? 1.0 / nv : 0.0;
#pragma unroll
    for (int t = 0; t < RPL; ++t) q[t][j] = kept[j] ? w[t] * inv : 0.0;
    R[j][j] = kept[j] ? nv : 0.0;
  }
#pragma unroll
  for (int t = 0; t < RPL; ++t)
    if (ok[t])
#pragma unroll
      for (int j = 0; j < RBM_K; ++j) Pt[(long long)(aa[t] * RBM_K + j) * F.N + pp[t]] = q[t][j];
  if (lane == 0) {
#pragma unroll
    for (int a = 0; a < RBM_K; ++a) {
#pragma unroll
      for (int b = 0; b < RBM_K; ++b) Nc[(long long)(a * RBM_K + b) * Cc.N + Kc] = R[a][b];
      ac[RBM_K * Kc + a] = kept[a] ? 1 : 0;
    }
  }
}

// Smoothed prolongator from the per-point tentative blocks:
// P[a, J] = Pt[a] [agg(a) = J] - omega D_a^-1 sum_{b ~ a, agg(b) = J} A_ab Pt[b]
template <int BF, int BC, int KIND>
__global__ void k_build_P_t(Lat F, Lat Cc, const double* __restrict__ val, const double* __restrict__ dinv,
                            const double* __restrict__ Pt, double omega, double* __restrict__ P) {
  const int R = St<KIND>::R;
  const int ns = p_slots(R);
  const int nslot = ns * ns * ns;
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= F.N * nslot) return;
  const int s = (int)(tid / F.N);
  const long long p = tid - (long long)s * F.N;
  int a, b, c;
  F.ijk(p, a, b, c);
  const int sx = s % ns, sy = (s / ns) % ns, sz = s / (ns * ns);
  const int I = p_lo(a, R) + sx, J = p_lo(b, R) + sy, K = p_lo(c, R) + sz;
  double out[BF * BC];
  for (int q = 0; q < BF * BC; ++q) out[q] = 0.0;
  if (Cc.in(I, J, K)) {
    double ap[BF * BC];
    for (int q = 0; q < BF * BC; ++q) ap[q] = 0.0;
    for (int o = 0; o < St<KIND>::N; ++o) {
      int dx, dy, dz;
      St<KIND>::off(o, dx, dy, dz);
      const int na = a + dx, nb = b + dy, nc = c + dz;
      if (!F.in(na, nb, nc)) continue;
      if (na / 3 != I || nb / 3 != J || nc / 3 != K) continue;
      const long long q = F.id(na, nb, nc);
      const double* v = val + (long long)o * BF * BF * F.N + p;
      for (int r = 0; r < BF; ++r)
        for (int t = 0; t < BC; ++t) {
          double z = 0.0;
          for (int u = 0; u < BF; ++u) z += v[(long long)(r * BF + u) * F.N] * Pt[(long long)(u * BC + t) * F.N + q];
          ap[r * BC + t] += z;
        }
    }
    for (int r = 0; r < BF; ++r)
      for (int t = 0; t < BC; ++t) {
        double z = 0.0;
        for (int u = 0; u < BF; ++u) z += dinv[(long long)(r * BF + u) * F.N + p] * ap[u * BC + t];
        out[r * BC + t] = -omega * z;
      }
    if (a / 3 == I && b / 3 == J && c / 3 == K)
      for (int q = 0; q < BF * BC; ++q) out[q] += Pt[(long long)q * F.N + p];
  }
  for (int q = 0; q < BF * BC; ++q) P[((long long)s * BF * BC + q) * F.N + p] = out[q];
}

// Galerkin faces -> cells: A_1[T, T'] = sum_{f in T, g} pw_f C_fg pw_g [T' adjacent to g]
__global__ void k_rap_faces(FaceTopo d, const int* __restrict__ col, const double* __restrict__ C,
                            const double* __restrict__ pw, double* __restrict__ A1, unsigned char* __restrict__ act) {
  const long long Tc = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (Tc >= d.nT) return;
  const int i = (int)(Tc % d.nx), j = (int)((Tc / d.nx) % d.ny), k = (int)(Tc / ((long long)d.nx * d.ny));
  double acc[25];
  for (int q = 0; q < 25; ++q) acc[q] = 0.0;
  bool any = false;
  for (int lf = 0; lf < 6; ++lf) {
    const long long f = ft_cell_face(d, i, j, k, lf);
    const double wf = pw[f];
    if (wf == 0.0) continue;
    any = true;
    for (int q = 0; q < 11; ++q) {
      const long long g = col[q * d.nF + f];
      const double v = C[q * d.nF + f];
      const double wg = pw[g];
      if (v == 0.0 || wg == 0.0) continue;
      int cc[2][3];
      const int cnt = ft_face_cells(d, g, cc);
      for (int e = 0; e < cnt; ++e) {
        const int o = St<ST_DIAMOND2>::idx(cc[e][0] - i, cc[e][1] - j, cc[e][2] - k);
        if (o >= 0) acc[o] += wf * v * wg;
      }
    }
  }
  act[Tc] = any ? 1 : 0;
  if (!any) acc[12] = 1.0;
  for (int q = 0; q < 25; ++q) A1[(long long)q * d.nT + Tc] = acc[q];
}

// ------------------------------------------------------------------ host helpers
// the face level's topology for the sweeps and transfers (32-bit: nF < 2^31)
FaceTopo32 face_topo(const Ctx& c) {
  if (c.nF >= (1LL << 31) / 11) throw Error{MHFP_ERR_ARG, "too many faces for 32-bit face indexing"};
  return FaceTopo32::make(c.nx, c.ny, c.nz, c.nT, c.nF, c.nFx, c.nFy);
}

// y = b - A x (y = A x when b is null) on a lattice level with schedule sched
template <typename T>
void launch_spmv(Ctx& c, const StructOp& A, int bs, const T* val, const T* x, const T* b, T* y, int sched) {
  sweep_spmv<T>(c.stream, A, bs, val, x, b, y, sched);
}

void level_spmv(Ctx& c, Level& L, const double* x, const double* b, double* y) {
  if (L.faces) {
    k_spmv_ell<double><<<lgrid(grid_for(L.n, 256)), 256, 0, c.stream>>>(face_topo(c), L.ell ? L.ell : c.Cpi, x, b, y,
                                                                         lbytes());
  } else {
    launch_spmv<double>(c, L.A, L.bs, L.A.val, x, b, y, default_schedule(L.A.N, L.bs));
  }
  MHFP_LAUNCH_CHECK();
}

void alloc_work(Ctx& c, Level& L) {
  L.x = dalloc_n<double>(c, L.n);
  L.b = dalloc_n<double>(c, L.n);
  L.r = dalloc_n<double>(c, L.n);
  L.d = dalloc_n<double>(c, L.n);
  L.y = dalloc_n<double>(c, L.n);
}

// rho(D^-1 A) by power iteration from the fixed start vector
double spectral_radius(Ctx& c, Level& L) {
  const long long n = L.n;
  double* v = L.x;
  double* w = L.y;
  k_power_start<<<grid_for(n, 256), 256, 0, c.stream>>>(n, v);
  MHFP_LAUNCH_CHECK();
  double nv = device_norm2(c, v, n);
  k_scale_by<<<grid_for(n, 256), 256, 0, c.stream>>>(n, 1.0 / nv, v);
  MHFP_LAUNCH_CHECK();
  double rho = 0.0;
  for (int it = 0; it < c.opt.power_iters; ++it) {
    level_spmv(c, L, v, nullptr, L.r);
    dispatch_bs(L.bs, [&](auto BS) {
      k_apply_dinv<BS.value><<<grid_for(L.npts, 256), 256, 0, c.stream>>>(L.npts, L.dinv, L.r, w);
    });
    MHFP_LAUNCH_CHECK();
    rho = device_norm2(c, w, n);
    k_scale_by<<<grid_for(n, 256), 256, 0, c.stream>>>(n, 1.0 / rho, w);
    MHFP_LAUNCH_CHECK();
    std::swap(v, w);
  }
  return rho;
}

// Gauss-Jordan inverse with partial pivoting (host, FP64), row-major
// Dense inverse of the coarsest level by Gauss-Jordan elimination on the GPU
// (FP64, augmented [A | I] of n x 2n, row-major).  The coarse operators are
// Galerkin products of SPD operators (Dirichlet rows carry a unit diagonal),
// so elimination needs no pivoting; a pivot that is not positive and finite
// sets *err and the host reports a singular level.  Column col takes two
// kernels: the first copies the scaled pivot row and the multipliers, the
// second updates every row from those copies (no read/write hazard).
__global__ void k_gj_pivot(int n, int col, const double* __restrict__ M, double* __restrict__ prow,
                           double* __restrict__ fcol, int* __restrict__ err) {
  const int w = 2 * n;
  const double piv = M[(long long)col * w + col];
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t == 0 && !(piv > 0.0 && piv < 1e300)) *err = 1;
  if (t < w) prow[t] = t < col ? 0.0 : M[(long long)col * w + t] / piv;
  if (t < n) fcol[t] = M[(long long)t * w + col];
}

__global__ void k_gj_update(int n, int col, double* __restrict__ M, const double* __restrict__ prow,
                            const double* __restrict__ fcol) {
  const int w = 2 * n;
  const int k = col + blockIdx.x * blockDim.x + threadIdx.x;
  const int r = blockIdx.y;
  if (k >= w) return;
  double* m = M + (long long)r * w + k;
  *m = (r == col) ? prow[k] : *m - fcol[r] * prow[k];
}

__global__ void k_gj_extract(int n, const double* __restrict__ M, double* __restrict__ inv) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * n) return;
  const long long r = t / n, cidx = t % n;
  inv[t] = M[r * 2 * n + n + cidx];
}

__global__ void k_gj_init(int n, const double* __restrict__ A, double* __restrict__ M) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * 2 * n) return;
  const long long r = t / (2 * n), cidx = t % (2 * n);
  M[t] = cidx < n ? A[r * n + cidx] : (cidx - n == r ? 1.0 : 0.0);
}

// A (host, n x n row-major) -> its inverse in device memory `inv`.  With
// keep, the elimination workspace is the handle's persistent one (allocated
// once, for permeability updates); otherwise it is allocated and freed here.
void invert_dense_gpu(Ctx& c, const std::vector<double>& A, int n, double* inv, bool keep = false) {
  double *dA = nullptr, *M = nullptr, *prow = nullptr, *fcol = nullptr;
  int* err = nullptr;
  auto release = [&] {
    if (keep) return;
    cudaFree(dA);
    cudaFree(M);
    cudaFree(prow);
    cudaFree(fcol);
    cudaFree(err);
  };
  cudaError_t e = cudaSuccess;
  if (keep) {
    if (c.gj_n < n) {
      c.gj_A = dalloc_n<double>(c, (size_t)n * n);
      c.gj_M = dalloc_n<double>(c, (size_t)n * 2 * n);
      c.gj_prow = dalloc_n<double>(c, (size_t)2 * n);
      c.gj_fcol = dalloc_n<double>(c, (size_t)n);
      if (!c.gj_err) c.gj_err = dalloc_n<int>(c, 1);
      c.gj_n = n;
    }
    dA = c.gj_A;
    M = c.gj_M;
    prow = c.gj_prow;
    fcol = c.gj_fcol;
    err = c.gj_err;
  } else {
    e = cudaMalloc(&dA, (size_t)n * n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&M, (size_t)n * 2 * n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&prow, (size_t)2 * n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&fcol, (size_t)n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(&err, sizeof(int));
  }
  if (e != cudaSuccess) {
    release();
    throw Error{MHFP_ERR_OOM, "device allocation failed (dense coarsest level)"};
  }
  try {
    MHFP_CUDA(cudaMemcpyAsync(dA, A.data(), (size_t)n * n * sizeof(double), cudaMemcpyHostToDevice, c.stream));
    MHFP_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c.stream));
    k_gj_init<<<grid_for((long long)n * 2 * n, 256), 256, 0, c.stream>>>(n, dA, M);
    MHFP_LAUNCH_CHECK();
    for (int col = 0; col < n; ++col) {
      k_gj_pivot<<<grid_for(2 * n, 256), 256, 0, c.stream>>>(n, col, M, prow, fcol, err);
      MHFP_LAUNCH_CHECK();
      k_gj_update<<<dim3(grid_for(2 * n - col, 256), n), 256, 0, c.stream>>>(n, col, M, prow, fcol);
      MHFP_LAUNCH_CHECK();
    }
    k_gj_extract<<<grid_for((long long)n * n, 256), 256, 0, c.stream>>>(n, M, inv);
    MHFP_LAUNCH_CHECK();
    int h_err = 0;
    MHFP_CUDA(cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    MHFP_CUDA(cudaStreamSynchronize(c.stream));
    if (h_err) throw Error{MHFP_ERR_ARG, "singular or indefinite coarsest multigrid level"};
  } catch (...) {
    cudaStreamSynchronize(c.stream);
    release();
    throw;
  }
  release();
}

void make_dense_coarse(Ctx& c, Level& L) {
  const int n = (int)L.n;
  std::vector<double> A((size_t)n * n, 0.0);
  if (L.faces) {
    std::vector<int> col(11 * (size_t)n);
    std::vector<double> val(11 * (size_t)n);
    MHFP_CUDA(cudaMemcpyAsync(col.data(), c.ell_col, col.size() * sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    MHFP_CUDA(cudaMemcpyAsync(val.data(), c.Cpi, val.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    MHFP_CUDA(cudaStreamSynchronize(c.stream));
    for (int f = 0; f < n; ++f)
      for (int q = 0; q < 11; ++q) A[(size_t)f * n + col[(size_t)q * n + f]] += val[(size_t)q * n + f];
  } else {
    const StructOp& S = L.A;
    const int bs = S.bs, no = S.noff();
    std::vector<double> val((size_t)no * bs * bs * S.N);
    MHFP_CUDA(cudaMemcpyAsync(val.data(), S.val, val.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    MHFP_CUDA(cudaStreamSynchronize(c.stream));
    for (long long p = 0; p < S.N; ++p) {
      const int i = (int)(p % S.Lx), j = (int)((p / S.Lx) % S.Ly), k = (int)(p / ((long long)S.Lx * S.Ly));
      for (int o = 0; o < no; ++o) {
        int dx, dy, dz;
        stencil_offset(S.kind, o, dx, dy, dz);
        const int a = i + dx, b = j + dy, cc = k + dz;
        if (a < 0 || a >= S.Lx || b < 0 || b >= S.Ly || cc < 0 || cc >= S.Lz) continue;
        const long long q = a + (long long)S.Lx * (b + (long long)S.Ly * cc);
        for (int r = 0; r < bs; ++r)
          for (int t = 0; t < bs; ++t)
            A[(size_t)(bs * p + r) * n + bs * q + t] += val[((size_t)o * bs * bs + r * bs + t) * S.N + p];
      }
    }
  }
  const bool rebuild = L.dense_inv != nullptr;
  if (!rebuild) L.dense_inv = dalloc_n<double>(c, (size_t)n * n);
  invert_dense_gpu(c, A, n, L.dense_inv, rebuild);
}

void finish_level(Ctx& c, Level& L) {
  if (!L.dinv) L.dinv = dalloc_n<double>(c, (size_t)L.bs * L.bs * L.npts);
  if (L.faces) {
    k_dinv_ell<<<grid_for(L.n, 256), 256, 0, c.stream>>>(L.n, L.ell ? L.ell : c.Cpi, L.dinv);
  } else {
    const Lat lat = lat_of(L.A);
    dispatch_bs(L.bs, [&](auto BS) {
      dispatch_kind_bs<BS.value>(L.A.kind, [&](auto K) {
        k_dinv<BS.value, K.value><<<grid_for(lat.N, 256), 256, 0, c.stream>>>(lat, L.A.val, L.dinv);
      });
    });
  }
  MHFP_LAUNCH_CHECK();
  L.lmax = 1.1 * spectral_radius(c, L);
}

// the transfer kernels index the prolongator [slot][entry][fine point] in
// 32-bit unsigned arithmetic: refuse levels where that would wrap
void check_transfer_index(long long rows, long long n) {
  if (rows * n >= (1LL << 32)) throw Error{MHFP_ERR_ARG, "level too large for 32-bit transfer indexing"};
}

// one smoothed-aggregation coarsening step of a lattice level.  With
// `into` (a permeability update), the next level already exists and its
// values, its activity mask and L's prolongator are recomputed in place,
// with the handle's persistent Galerkin scratch.
Level coarsen(Ctx& c, Level& L, Level* into = nullptr) {
  const StructOp& A = L.A;
  const int R = stencil_radius(A.kind);
  L.R = R;
  L.cbs = L.bs;
  Level Cl;
  if (into) Cl = *into;
  Cl.bs = L.bs;
  Cl.A.Lx = (A.Lx + 2) / 3; Cl.A.Ly = (A.Ly + 2) / 3; Cl.A.Lz = (A.Lz + 2) / 3;
  Cl.A.N = (long long)Cl.A.Lx * Cl.A.Ly * Cl.A.Lz;
  Cl.A.bs = L.bs;
  Cl.A.kind = (R == 1) ? ST_BOX1 : ST_BOX2;
  Cl.npts = Cl.A.N;
  Cl.n = Cl.A.N * L.bs;
  Cl.R = stencil_radius(Cl.A.kind);
  const Lat F = lat_of(A), Cc = lat_of(Cl.A);
  const int ns = p_slots(R), nq = q_slots(R);
  const int bs2 = L.bs * L.bs;
  check_transfer_index((long long)ns * ns * ns * bs2, F.N);
  if (!L.P) L.P = dalloc_n<double>(c, (size_t)ns * ns * ns * bs2 * F.N);
  if (!Cl.active) Cl.active = dalloc_n<unsigned char>(c, Cl.n);
  if (!Cl.A.val) Cl.A.val = dalloc_n<double>(c, (size_t)Cl.A.noff() * bs2 * Cc.N);
  const size_t q_elems = (size_t)nq * nq * nq * bs2 * F.N;
  double* Q = nullptr;
  if (into) {
    if (c.upd_Q_elems < q_elems) {
      c.upd_Q = dalloc_n<double>(c, q_elems);
      c.upd_Q_elems = q_elems;
    }
    Q = c.upd_Q;
  } else {
    MHFP_CUDA(cudaMalloc(&Q, q_elems * sizeof(double)));
  }
  const double omega = 4.0 / (3.0 * L.lmax);
  try {
    dispatch_bs13(L.bs, [&](auto BS) {
      dispatch_kind_bs<BS.value>(A.kind, [&](auto K) {
        k_build_P<BS.value, K.value><<<grid_for(F.N * ns * ns * ns, 256), 256, 0, c.stream>>>(F, Cc, A.val, L.dinv,
                                                                                             L.active, omega, L.P);
        MHFP_LAUNCH_CHECK();
        k_active_coarse<BS.value><<<grid_for(Cc.N, 256), 256, 0, c.stream>>>(F, Cc, L.active, Cl.active);
        MHFP_LAUNCH_CHECK();
        k_build_Q<BS.value, BS.value, K.value><<<grid_for(F.N * nq * nq * nq, 256), 256, 0, c.stream>>>(F, Cc, A.val,
                                                                                                     L.P, Q);
        MHFP_LAUNCH_CHECK();
      });
      // coarse levels of the 27-point displacement lattice stay 27-point; the
      // scalar levels become 125-point
      if constexpr (BS.value == 3)
        k_rap<BS.value, BS.value, ST_BOX1><<<grid_for(Cc.N * 27, 128), 128, 0, c.stream>>>(F, Cc, R, L.P, Q,
                                                                                           Cl.active, Cl.A.val);
      else
        k_rap<BS.value, BS.value, ST_BOX2><<<grid_for(Cc.N * 125, 128), 128, 0, c.stream>>>(F, Cc, R, L.P, Q,
                                                                                             Cl.active, Cl.A.val);
      MHFP_LAUNCH_CHECK();
    });
    MHFP_CUDA(cudaStreamSynchronize(c.stream));
  } catch (...) {
    if (!into) cudaFree(Q);
    throw;
  }
  if (!into) MHFP_CUDA(cudaFree(Q));
  return Cl;
}

void build_u_level0(Ctx& c) {
  c.hu.clear();
  Level L0;
  L0.bs = 3;
  L0.A = c.Auu;
  L0.npts = c.nN;
  L0.n = c.nU;
  L0.R = 1;
  L0.active = dalloc_n<unsigned char>(c, c.nU);
  {
    std::vector<unsigned char> fix(c.nN), act(c.nU);
    MHFP_CUDA(cudaMemcpyAsync(fix.data(), c.node_fix, c.nN, cudaMemcpyDeviceToHost, c.stream));
    MHFP_CUDA(cudaStreamSynchronize(c.stream));
    for (long long n = 0; n < c.nN; ++n)
      for (int q = 0; q < 3; ++q) act[3 * n + q] = ((fix[n] >> q) & 1) ? 0 : 1;
    MHFP_CUDA(cudaMemcpyAsync(L0.active, act.data(), c.nU, cudaMemcpyHostToDevice, c.stream));
    MHFP_CUDA(cudaStreamSynchronize(c.stream));
  }
  c.hu.push_back(L0);
}

void build_u(Ctx& c) {
  build_u_level0(c);
  while (c.hu.back().npts > c.opt.coarse_max && c.hu.size() < 8) {
    Level& L = c.hu.back();
    alloc_work(c, L);
    finish_level(c, L);
    Level Cl = coarsen(c, L);
    c.hu.push_back(Cl);
  }
  Level& last = c.hu.back();
  alloc_work(c, last);
  make_dense_coarse(c, last);
}

// The displacement hierarchy of M_III^(h): the same aggregates, with the six
// rigid-body modes as the near-kernel.  Level 0 is A_uu (3 dofs per node);
// every coarse point carries 6 dofs (a mode its aggregate cannot represent
// leaves an inactive dof with a unit diagonal).  P = (I - omega D^-1 A) P_t
// with P_t the Gram-Schmidt factors of the aggregates, Galerkin coarse
// operators in the same two gather passes as M_II^(h).
void build_u_rbm(Ctx& c) {
  build_u_level0(c);
  // centroid of the nodes (the rotations' axis point), summed in node order
  double cen[3] = {0, 0, 0};
  {
    std::vector<double> xyz(3 * c.nN);
    MHFP_CUDA(cudaMemcpyAsync(xyz.data(), c.coords, xyz.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    MHFP_CUDA(cudaStreamSynchronize(c.stream));
    for (long long p = 0; p < c.nN; ++p)
      for (int a = 0; a < 3; ++a) cen[a] += xyz[3 * p + a];
    for (int a = 0; a < 3; ++a) cen[a] /= (double)c.nN;
  }
  const double* Nprev = nullptr;
  while (c.hu.back().npts > c.opt.coarse_max && c.hu.size() < 8) {
    Level& L = c.hu.back();
    alloc_work(c, L);
    finish_level(c, L);
    const int BFv = L.bs;
    const StructOp& A = L.A;
    L.R = 1;
    L.cbs = RBM_K;
    Level Cl;
    Cl.bs = RBM_K;
    Cl.A.Lx = (A.Lx + 2) / 3; Cl.A.Ly = (A.Ly + 2) / 3; Cl.A.Lz = (A.Lz + 2) / 3;
    Cl.A.N = (long long)Cl.A.Lx * Cl.A.Ly * Cl.A.Lz;
    Cl.A.bs = RBM_K;
    Cl.A.kind = ST_BOX1;
    Cl.npts = Cl.A.N;
    Cl.n = Cl.A.N * RBM_K;
    Cl.R = 1;
    const Lat F = lat_of(A), Cc = lat_of(Cl.A);
    const int ns = p_slots(1), nq = q_slots(1);
    const int pb = BFv * RBM_K;
    double* Pt = dalloc_n<double>(c, (size_t)pb * F.N);
    double* Nc = dalloc_n<double>(c, (size_t)RBM_K * RBM_K * Cc.N);
    Cl.active = dalloc_n<unsigned char>(c, Cl.n);
    check_transfer_index((long long)ns * ns * ns * pb, F.N);
    L.P = dalloc_n<double>(c, (size_t)ns * ns * ns * pb * F.N);
    Cl.A.val = dalloc_n<double>(c, (size_t)27 * RBM_K * RBM_K * Cc.N);
    MHFP_CUDA(cudaMemsetAsync(Pt, 0, (size_t)pb * F.N * sizeof(double), c.stream));
    const double omega = 4.0 / (3.0 * L.lmax);
    double* Q = nullptr;
    MHFP_CUDA(cudaMalloc(&Q, (size_t)nq * nq * nq * pb * F.N * sizeof(double)));
    try {
      const unsigned warps = grid_for(Cc.N * 32, 128);
      auto galerkin = [&](auto BF) {
        constexpr int bf = decltype(BF)::value;
        k_build_P_t<bf, RBM_K, ST_BOX1><<<grid_for(F.N * ns * ns * ns, 256), 256, 0, c.stream>>>(F, Cc, A.val, L.dinv,
                                                                                                 Pt, omega, L.P);
        MHFP_LAUNCH_CHECK();
        k_build_Q<bf, RBM_K, ST_BOX1><<<grid_for(F.N * nq * nq * nq, 256), 256, 0, c.stream>>>(F, Cc, A.val, L.P, Q);
        MHFP_LAUNCH_CHECK();
        k_rap<bf, RBM_K, ST_BOX1><<<grid_for(Cc.N * 27, 128), 128, 0, c.stream>>>(F, Cc, 1, L.P, Q, Cl.active,
                                                                                   Cl.A.val);
        MHFP_LAUNCH_CHECK();
      };
      if (BFv == 3) {
        k_rbm_tentative<3, 3><<<warps, 128, 0, c.stream>>>(F, Cc, c.coords, L.active, nullptr, cen[0], cen[1], cen[2],
                                                           Pt, Nc, Cl.active);
        MHFP_LAUNCH_CHECK();
        galerkin(std::integral_constant<int, 3>{});
      } else {
        k_rbm_tentative<RBM_K, 6><<<warps, 128, 0, c.stream>>>(F, Cc, c.coords, L.active, Nprev, cen[0], cen[1],
                                                               cen[2], Pt, Nc, Cl.active);
        MHFP_LAUNCH_CHECK();
        galerkin(std::integral_constant<int, RBM_K>{});
      }
      MHFP_CUDA(cudaStreamSynchronize(c.stream));
    } catch (...) {
      cudaFree(Q);
      throw;
    }
    MHFP_CUDA(cudaFree(Q));
    Nprev = Nc;
    c.hu.push_back(Cl);
  }
  Level& last = c.hu.back();
  alloc_work(c, last);
  make_dense_coarse(c, last);
}

void build_pi(Ctx& c) {
  c.hpi.clear();
  Level L0;
  L0.faces = true;
  L0.bs = 1;
  L0.npts = c.nF;
  L0.n = c.nF;
  c.hpi.push_back(L0);
  if (c.nF <= c.opt.coarse_max) {
    alloc_work(c, c.hpi.back());
    make_dense_coarse(c, c.hpi.back());
    return;
  }
  {
    Level& F = c.hpi.back();
    alloc_work(c, F);
    finish_level(c, F);
    Level L1;
    L1.bs = 1;
    L1.A.Lx = c.nx; L1.A.Ly = c.ny; L1.A.Lz = c.nz;
    L1.A.N = c.nT; L1.A.bs = 1; L1.A.kind = ST_DIAMOND2;
    L1.npts = c.nT; L1.n = c.nT; L1.R = 2;
    L1.A.val = dalloc_n<double>(c, (size_t)25 * c.nT);
    L1.active = dalloc_n<unsigned char>(c, c.nT);
    k_rap_faces<<<grid_for(c.nT, 128), 128, 0, c.stream>>>(FaceTopo{c.nx, c.ny, c.nz, c.nT, c.nF, c.nFx, c.nFy},
                                                           c.ell_col, c.Cpi, c.pw, L1.A.val, L1.active);
    MHFP_LAUNCH_CHECK();
    c.hpi.push_back(L1);
  }
  while (c.hpi.back().npts > c.opt.coarse_max && c.hpi.size() < 8) {
    Level& L = c.hpi.back();
    alloc_work(c, L);
    finish_level(c, L);
    Level Cl = coarsen(c, L);
    c.hpi.push_back(Cl);
  }
  Level& last = c.hpi.back();
  alloc_work(c, last);
  make_dense_coarse(c, last);
}

// ------------------------------------------------------------------ V-cycle
// Pointers of one level in the precision T of the cycle: the FP64 arrays
// built by the set-up, or their FP32 copies for the mixed-precision cycle.
template <typename T>
struct LV {
  const T *val, *dinv, *P, *ell, *pw;
  T *r, *d, *y;
};
LV<double> view(Ctx& c, Level& L, double) {
  return {L.A.val, L.dinv, L.P, L.ell ? L.ell : c.Cpi, c.pw, L.r, L.d, L.y};
}
LV<float> view(Ctx& c, Level& L, float) { return {L.valf, L.dinvf, L.Pf, c.Cpif, c.pwf, L.rf, L.df, L.yf}; }
double* bvec(Level& L, double) { return L.b; }
float* bvec(Level& L, float) { return L.bf; }
double* xvec(Level& L, double) { return L.x; }
float* xvec(Level& L, float) { return L.xf; }

template <typename T>
void level_spmv_t(Ctx& c, Level& L, const T* x, const T* b, T* y) {
  const LV<T> v = view(c, L, T());
  if (L.faces) {
    k_spmv_ell<T><<<lgrid(grid_for(L.n, 256)), 256, 0, c.stream>>>(face_topo(c), v.ell, x, b, y, lbytes());
  } else {
    launch_spmv<T>(c, L.A, L.bs, v.val, x, b, y, L.tpp ? L.tpp : default_schedule(L.A.N, L.bs));
  }
  MHFP_LAUNCH_CHECK();
}

// one Chebyshev sweep on a lattice level with schedule sched (the first
// sweep from zero has no stencil work and always runs one point per thread)
template <typename T>
void launch_cheb(Ctx& c, Level& L, const LV<T>& v, const T* b, const T* xin, T* out, T cd, T cr, int sched) {
  if (!xin) {
    sweep_cheb_zero<T>(c.stream, L.A.N, L.bs, v.dinv, b, out, v.d, cr);
    return;
  }
  sweep_cheb<T>(c.stream, L.A, L.bs, v.val, v.dinv, b, xin, out, v.d, cd, cr, sched);
}

// The symmetric FP32 sweep and residual of the finest displacement level
// with L.tpp resident blocks per SM (6 or 8; 0: 8 when one wave of 8 blocks
// of 256 per SM covers the level, else 6).
// schedule of the finest FP32 displacement level: 6 or 8 resident blocks of
// 256 threads per SM (0: 8 when one wave of 8 blocks per SM covers the
// level, else 6)
int sym_minb(const Level& L) {
  if (L.tpp >= 4 && L.tpp <= 8) return L.tpp;
  return L.A.N <= 152LL * 8 * 256 ? 8 : 6;
}

// the bulk-copy-fed variant (schedule 4): persistent CTAs, 4 per SM
void launch_sym_tma(Ctx& c, const Level& L, bool cheb, const float* b, const float* xin, float* xout, float* d,
                    float cd, float cr) {
  const Lat lat = lat_of(L.A);
  if (lat.N >= (1LL << 31) - TMA_NB) throw Error{MHFP_ERR_ARG, "level too large for the bulk-copy sweep"};
  const long long nblocks = (lat.N + TMA_NB - 1) / TMA_NB;
  const unsigned grid = (unsigned)std::min<long long>(nblocks, 3LL * c.n_sm);
  static bool attr = false;  // the dynamic shared memory above 48 KB, once per process
  if (!attr) {
    MHFP_CUDA(cudaFuncSetAttribute(k_sym_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TMA_SMEM));
    MHFP_CUDA(cudaFuncSetAttribute(k_sym_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TMA_SMEM));
    attr = true;
  }
  TmaSweep a{L.symf, L.dinvf, b, xin, xout, d, cd, cr, c.d_flag};
  if (cheb) k_sym_tma<true><<<lgrid(grid), TMA_THREADS, TMA_SMEM, c.stream>>>(lat, a, lbytes());
  else k_sym_tma<false><<<lgrid(grid), TMA_THREADS, TMA_SMEM, c.stream>>>(lat, a, lbytes());
}
void launch_cheb_sym(Ctx& c, const Level& L, const float* b, const float* xin, float* xout, float* d, float cd,
                     float cr) {
  const Lat lat = lat_of(L.A);
  if (!xin) {  // the first step from zero has no stencil work
    sweep_cheb_zero<float>(c.stream, lat.N, 3, L.dinvf, b, xout, d, cr);
    MHFP_LAUNCH_CHECK();
    return;
  }
  const int mb = sym_minb(L);
  if (mb == 4)
    launch_sym_tma(c, L, true, b, xin, xout, d, cd, cr);
  else if (mb == 5)
    k_cheb_u0_sym<float, 5><<<lgrid(grid_for(lat.N, 256)), 256, 0, c.stream>>>(lat, L.symf, L.dinvf, b, xin,
                                                                                xout, d, cd, cr, lbytes());
  else if (mb == 7)
    k_cheb_u0_sym<float, 7><<<lgrid(grid_for(lat.N, 256)), 256, 0, c.stream>>>(lat, L.symf, L.dinvf, b, xin,
                                                                                xout, d, cd, cr, lbytes());
  else if (mb == 8)
    k_cheb_u0_sym<float, 8><<<lgrid(grid_for(lat.N, 256)), 256, 0, c.stream>>>(lat, L.symf, L.dinvf, b, xin,
                                                                                xout, d, cd, cr, lbytes());
  else
    k_cheb_u0_sym<float, 6><<<lgrid(grid_for(lat.N, 256)), 256, 0, c.stream>>>(lat, L.symf, L.dinvf, b, xin,
                                                                                xout, d, cd, cr, lbytes());
  MHFP_LAUNCH_CHECK();
}
void launch_resid_sym(Ctx& c, const Level& L, const float* x, const float* b, float* y) {
  const Lat lat = lat_of(L.A);
  const int mb = sym_minb(L);
  if (mb == 4)
    launch_sym_tma(c, L, false, b, x, y, nullptr, 0.f, 0.f);
  else if (mb == 5)
    k_resid_u0_sym<float, 5><<<lgrid(grid_for(lat.N, 256)), 256, 0, c.stream>>>(lat, L.symf, x, b, y,
                                                                                 lbytes());
  else if (mb == 7)
    k_resid_u0_sym<float, 7><<<lgrid(grid_for(lat.N, 256)), 256, 0, c.stream>>>(lat, L.symf, x, b, y,
                                                                                 lbytes());
  else if (mb == 8)
    k_resid_u0_sym<float, 8><<<lgrid(grid_for(lat.N, 256)), 256, 0, c.stream>>>(lat, L.symf, x, b, y,
                                                                                 lbytes());
  else
    k_resid_u0_sym<float, 6><<<lgrid(grid_for(lat.N, 256)), 256, 0, c.stream>>>(lat, L.symf, x, b, y,
                                                                                 lbytes());
  MHFP_LAUNCH_CHECK();
}

// Device time of one call of `body` (which enqueues kernels on c.stream):
// `reps` calls captured once into a CUDA graph on a private stream, the
// graph replayed once to warm up and three times under events, the fastest
// replay kept.  Timing graph replays leaves out host launch overhead, as in
// the solve, which runs as graphs.
template <class F>
float graph_time_us(Ctx& c, int reps, F&& body) {
  cudaStream_t user = c.stream, st = nullptr;
  MHFP_CUDA(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  MHFP_CUDA(cudaStreamSynchronize(user));
  const long long l0 = g_launches;
  cudaGraph_t g = nullptr;
  cudaGraphExec_t ge = nullptr;
  c.stream = st;
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    try {
      for (int r = 0; r < reps; ++r) body();
    } catch (...) {
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      c.stream = user;
      cudaStreamDestroy(st);
      throw;
    }
    e = cudaStreamEndCapture(st, &g);
  }
  c.stream = user;
  g_launches = l0;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
  if (g) cudaGraphDestroy(g);
  float best = 1e30f;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  for (int it = 0; it < 4 && e == cudaSuccess; ++it) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = cudaGraphLaunch(ge, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && it > 0 && ms < best) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (ge) cudaGraphExecDestroy(ge);
  cudaStreamDestroy(st);
  MHFP_CUDA(e);
  return best * 1e3f / reps;
}

// Set-up autotuner for the finest displacement level in FP32: time the two
// occupancy variants of the symmetric sweep and keep the faster in L.tpp.
void autotune_fine_sym(Ctx& c, Level& L) {
  MHFP_CUDA(cudaMemsetAsync(L.bf, 0, L.n * sizeof(float), c.stream));
  MHFP_CUDA(cudaMemsetAsync(L.xf, 0, L.n * sizeof(float), c.stream));
  MHFP_CUDA(cudaMemsetAsync(L.df, 0, L.n * sizeof(float), c.stream));
  float best = 1e30f;
  int best_minb = 0;
  for (int minb : {8, 7, 6, 5, 4}) {
    L.tpp = minb;
    const float us = graph_time_us(c, 5, [&] { launch_cheb_sym(c, L, L.bf, L.xf, L.yf, L.df, 0.5f, 0.5f); });
    if (us < best) {
      best = us;
      best_minb = minb;
    }
  }
  L.tpp = best_minb;
  L.sweep_us = best;
}

// Set-up autotuner: time the launch schedules of a coarse level's Chebyshev
// sweep (one point per thread; offsets split over 4, 8 or 16 warps: same
// arithmetic up to the order of the partial sums) and keep the fastest for
// this level's sweeps and residuals.
template <typename T>
void autotune_level(Ctx& c, Level& L) {
  const LV<T> v = view(c, L, T());
  T* b = bvec(L, T());
  T* x = xvec(L, T());
  MHFP_CUDA(cudaMemsetAsync(b, 0, L.n * sizeof(T), c.stream));
  MHFP_CUDA(cudaMemsetAsync(x, 0, L.n * sizeof(T), c.stream));
  MHFP_CUDA(cudaMemsetAsync(v.d, 0, L.n * sizeof(T), c.stream));
  float best = 1e30f;
  int best_tpp = default_schedule(L.A.N, L.bs);
  for (int tpp : {1, 4, 8, 16}) {
    const float us = graph_time_us(c, 10, [&] {
      launch_cheb<T>(c, L, v, b, x, v.y, T(0.5), T(0.5), tpp);
      MHFP_LAUNCH_CHECK();
    });
    if (us < best) {
      best = us;
      best_tpp = tpp;
    }
  }
  L.tpp = best_tpp;
  L.sweep_us = best;
}

// Chebyshev smoothing of level l from x0 (null: from zero) into dst.  Each
// step reads neighbours of its input, so it cannot update in place: the
// steps write dst and alt in turn, chosen so that the last one writes dst
// (the first step's output differs from x0 when alt is the buffer that x0
// is not, or x0 is null).
// the centre of level L's Chebyshev interval [lmax / ratio, lmax]
double cheb_theta(const Ctx& c, const Level& L) {
  const double lmax = L.lmax, lmin = lmax / c.opt.cheb_ratio;
  return 0.5 * (lmax + lmin);
}

// output buffer of step s of a smoothing into dst that alternates with alt
template <typename T>
T* step_out(int deg, int s, T* dst, T* alt) {
  return ((deg - 1 - s) % 2 == 0) ? dst : alt;
}

// With first_done the first step (from zero, x0 null) was already taken by
// the restriction that produced b (its output in that step's buffer, its
// direction in the level's d): the smoothing goes on from the second step.
template <typename T>
void smooth(Ctx& c, std::vector<Level>& H, int l, const T* b, const T* x0, T* dst, T* alt, bool time_it,
            bool first_done = false) {
  Level& L = H[l];
  const LV<T> v = view(c, L, T());
  const int deg = c.opt.cheb_degree;
  const double lmax = L.lmax, lmin = lmax / c.opt.cheb_ratio;
  const double theta = cheb_theta(c, L), delta = 0.5 * (lmax - lmin), sigma = theta / delta;
  double rho = 1.0 / sigma;
  const T* xin = first_done ? step_out(deg, 0, dst, alt) : x0;
  for (int s = first_done ? 1 : 0; s < deg; ++s) {
    T* out = step_out(deg, s, dst, alt);
    double cd = 0.0, cr = 1.0 / theta;
    if (s > 0) {
      const double rn = 1.0 / (2.0 * sigma - rho);
      cd = rn * rho;
      cr = 2.0 * rn / delta;
      rho = rn;
    }
    if (time_it && xin) timing_begin(c, 0);
    if (L.faces) {
      k_cheb_ell<T><<<lgrid(grid_for(L.n, 256)), 256, 0, c.stream>>>(face_topo(c), v.ell, v.dinv, b, xin, out, v.d,
                                                                     (T)cd, (T)cr, lbytes());
    } else if (time_it) {
      if constexpr (std::is_same<T, float>::value) {
        launch_cheb_sym(c, L, b, xin, out, v.d, (T)cd, (T)cr);
      } else {
        const Lat lat = lat_of(L.A);
        k_cheb_u0<T><<<lgrid(grid_for(lat.N, 256)), 256, 0, c.stream>>>(lat, v.val, v.dinv, b, xin, out, v.d, (T)cd,
                                                                         (T)cr, lbytes());
      }
    } else {
      launch_cheb<T>(c, L, v, b, xin, out, (T)cd, (T)cr, L.tpp ? L.tpp : default_schedule(L.A.N, L.bs));
    }
    MHFP_LAUNCH_CHECK();
    // algorithmic bytes of a Chebyshev sweep: the matrix values (27 blocks
    // per node in FP64, the 14 stored blocks of the symmetric FP32 copy) and
    // the 3x3 inverse diagonal per node, b, x_in, x_out and d read/written
    const double blocks = std::is_same<T, float>::value ? 14.0 : 27.0;
    if (time_it && xin) timing_end(c, 0, (blocks * 9 + 9) * sizeof(T) * L.npts + 5.0 * sizeof(T) * L.n);
    xin = out;
  }
}

template <typename T>
void vcycle_level(Ctx& c, std::vector<Level>& H, int l, const T* b, T* x, bool pre_done = false) {
  Level& L = H[l];
  const LV<T> v = view(c, L, T());
  if (L.dense_inv) {
    const int n = (int)L.n;
    k_dense_mv<T><<<lgrid((n + 1) / 2), 256, 0, c.stream>>>(n, L.dense_inv, b, x, lbytes());
    MHFP_LAUNCH_CHECK();
    return;
  }
  const bool fine_u = (&H == &c.hu) && l == 0;
  // the pre-smoothed and corrected iterate lives in s_buf, chosen so that the
  // post-smoothing's last step writes x: the level's other work vector when
  // the degree is odd, x itself when it is even (no copy back)
  T* s_buf = (c.opt.cheb_degree % 2 == 1) ? v.y : x;
  smooth<T>(c, H, l, b, nullptr, s_buf, s_buf == x ? v.y : x, fine_u, pre_done);
  if (fine_u) {
    if constexpr (std::is_same<T, float>::value) {
      launch_resid_sym(c, L, s_buf, b, v.r);
    } else {
      const Lat lat = lat_of(L.A);
      k_resid_u0<T><<<lgrid(grid_for(lat.N, 256)), 256, 0, c.stream>>>(lat, v.val, s_buf, b, v.r, lbytes());
      MHFP_LAUNCH_CHECK();
    }
  } else {
    level_spmv_t<T>(c, L, s_buf, b, v.r);
  }
  Level& C = H[l + 1];
  T* cb = bvec(C, T());
  T* cx = xvec(C, T());
  // the restriction also takes the coarse level's first Chebyshev step from
  // zero (d = cr D^-1 b into that step's buffer), unless it is the dense one
  const bool fuse = !C.dense_inv;
  const LV<T> cv = view(c, C, T());
  const int deg = c.opt.cheb_degree;
  T* cs_buf = (deg % 2 == 1) ? cv.y : cx;
  const T* fdinv = fuse ? cv.dinv : nullptr;
  const T fcr = fuse ? (T)(1.0 / cheb_theta(c, C)) : T(0);
  T* fx = fuse ? step_out(deg, 0, cs_buf, cs_buf == cx ? cv.y : cx) : nullptr;
  T* fd = fuse ? cv.d : nullptr;
  if (L.faces) {
    k_restrict_faces<T><<<lgrid(grid_for(c.nT, 256)), 256, 0, c.stream>>>(face_topo(c), v.pw, v.r, cb, fdinv, fcr,
                                                                          fx, fd, lbytes());
  } else {
    const Lat32 F = lat32_of(L.A), Cc = lat32_of(C.A);
    dispatch_pair(L.bs, C.bs, [&](auto BF, auto BC) {
      dispatch_r(L.R, [&](auto RR) {
        k_restrict_f<BF.value, BC.value, RR.value, T><<<lgrid(grid_for(C.A.N * 32, 256)), 256, 0, c.stream>>>(
            F, Cc, v.P, v.r, cb, fdinv, fcr, fx, fd, lbytes());
      });
    });
  }
  MHFP_LAUNCH_CHECK();
  vcycle_level<T>(c, H, l + 1, cb, cx, fuse);
  if (L.faces) {
    k_prolong_faces<T><<<lgrid(grid_for(c.nF, 256)), 256, 0, c.stream>>>(face_topo(c), v.pw, cx, s_buf, lbytes());
  } else {
    // one fine point per thread on large levels, slots split over 8 warps on small ones
    const Lat32 F = lat32_of(L.A), Cc = lat32_of(C.A);
    dispatch_pair(L.bs, C.bs, [&](auto BF, auto BC) {
      dispatch_r(L.R, [&](auto RR) {
        if (L.A.N >= 65536)
          k_prolong_f<BF.value, BC.value, RR.value, T><<<lgrid(grid_for(L.A.N, 256)), 256, 0, c.stream>>>(
              F, Cc, v.P, cx, s_buf, lbytes());
        else
          k_prolong_w<BF.value, BC.value, RR.value, 8, T><<<lgrid(grid_for(L.A.N, 32)), dim3(32, 8), 0, c.stream>>>(
              F, Cc, v.P, cx, s_buf, lbytes());
      });
    });
  }
  MHFP_LAUNCH_CHECK();
  smooth<T>(c, H, l, b, s_buf, x, v.y, fine_u);
}

float* cast_copy(Ctx& c, const double* src, size_t n) {
  float* d = dalloc_n<float>(c, n);
  k_cast_f32<<<grid_for((long long)n, 256), 256, 0, c.stream>>>((long long)n, src, d);
  MHFP_LAUNCH_CHECK();
  return d;
}

// FP32 copies of a hierarchy built in FP64 (the last level keeps its FP64
// dense inverse).  With fine_sym, level 0 (the finest displacement level,
// 27-point 3x3-block stencil) keeps only its symmetric half: the diagonal
// block and the 13 offsets after it, the last 14 x 9 x N values of the
// offset-major FP64 array.
void make_fp32(Ctx& c, std::vector<Level>& H, bool fine_sym) {
  for (size_t l = 0; l < H.size(); ++l) {
    Level& L = H[l];
    const size_t bs2 = (size_t)L.bs * L.bs;
    if (fine_sym && l == 0 && !L.dense_inv) {
      const long long N = L.A.N;
      // node-blocked: ceil(N / 32) blocks of 126 x 32 values, plus 8 zeroed
      // blocks that the bulk-copy sweep's last node block reads past the end
      const size_t sym_elems = (size_t)((N + 31) / 32 + TMA_NW) * 126 * 32;
      L.symf = dalloc_n<float>(c, sym_elems);
      MHFP_CUDA(cudaMemsetAsync(L.symf, 0, sym_elems * sizeof(float), c.stream));
      k_cast_f32_sym<<<grid_for(126 * N, 256), 256, 0, c.stream>>>(N, L.A.val + 13 * 9 * N, L.symf);
      MHFP_LAUNCH_CHECK();
    } else if (!L.faces) {
      L.valf = cast_copy(c, L.A.val, (size_t)L.A.noff() * bs2 * L.A.N);
    }
    if (L.dinv) L.dinvf = cast_copy(c, L.dinv, bs2 * L.npts);
    if (L.P) {
      const int ns = p_slots(L.R);
      L.Pf = cast_copy(c, L.P, (size_t)ns * ns * ns * L.bs * L.cbs * L.npts);
    }
    L.xf = dalloc_n<float>(c, L.n);
    L.bf = dalloc_n<float>(c, L.n);
    L.rf = dalloc_n<float>(c, L.n);
    L.df = dalloc_n<float>(c, L.n);
    L.yf = dalloc_n<float>(c, L.n);
  }
}

}  // namespace

void build_hierarchies(Ctx& c) {
  if (c.opt.near_kernel == 1) build_u_rbm(c);
  else build_u(c);
  build_pi(c);
  if (c.opt.precision == 1) {
    make_fp32(c, c.hu, true);
    make_fp32(c, c.hpi, false);
    c.Cpif = cast_copy(c, c.Cpi, (size_t)11 * c.nF);
    c.pwf = cast_copy(c, c.pw, c.nF);
  }
  if (c.opt.autotune) {
    // the finest displacement level runs k_cheb_u0 (FP64) or the symmetric
    // FP32 sweep, whose two occupancy variants are timed; tune the others
    // (schedules fixed by the options are not tuned)
    if (c.opt.precision == 1 && !c.hu[0].dense_inv && !c.opt.fine_blocks) autotune_fine_sym(c, c.hu[0]);
    for (auto* H : {&c.hu, &c.hpi})
      for (size_t l = 0; l < H->size(); ++l) {
        Level& L = (*H)[l];
        if (L.faces || L.dense_inv || (H == &c.hu && l == 0) || c.opt.schedule) continue;
        if (c.opt.precision == 1) autotune_level<float>(c, L);
        else autotune_level<double>(c, L);
      }
  }
  // schedules forced by the options
  if (c.opt.fine_blocks && c.opt.precision == 1 && !c.hu[0].dense_inv) c.hu[0].tpp = c.opt.fine_blocks;
  if (c.opt.schedule)
    for (auto* H : {&c.hu, &c.hpi})
      for (size_t l = 0; l < H->size(); ++l) {
        Level& L = (*H)[l];
        if (!L.faces && !L.dense_inv && !(H == &c.hu && l == 0)) L.tpp = c.opt.schedule;
      }
}

// The interface-pressure hierarchy after a permeability update: C~_pi has
// new values on the same pattern, so every level keeps its size, buffers
// and launch schedule; the diagonal inverses, lmax, prolongators, Galerkin
// products, dense coarsest inverse and FP32 copies are recomputed in place.
void rebuild_pi_hierarchy(Ctx& c) {
  auto& H = c.hpi;
  if (H.size() == 1) {
    make_dense_coarse(c, H[0]);
  } else {
    finish_level(c, H[0]);
    Level& L1 = H[1];
    k_rap_faces<<<grid_for(c.nT, 128), 128, 0, c.stream>>>(FaceTopo{c.nx, c.ny, c.nz, c.nT, c.nF, c.nFx, c.nFy},
                                                           c.ell_col, c.Cpi, c.pw, L1.A.val, L1.active);
    MHFP_LAUNCH_CHECK();
    for (size_t l = 1; l + 1 < H.size(); ++l) {
      finish_level(c, H[l]);
      H[l + 1] = coarsen(c, H[l], &H[l + 1]);
    }
    make_dense_coarse(c, H.back());
  }
  if (c.opt.precision == 1) {
    auto recast = [&](float* dst, const double* src, size_t n) {
      k_cast_f32<<<grid_for((long long)n, 256), 256, 0, c.stream>>>((long long)n, src, dst);
      MHFP_LAUNCH_CHECK();
    };
    for (Level& L : H) {
      const size_t bs2 = (size_t)L.bs * L.bs;
      if (!L.faces && L.valf) recast(L.valf, L.A.val, (size_t)L.A.noff() * bs2 * L.A.N);
      if (L.dinv && L.dinvf) recast(L.dinvf, L.dinv, bs2 * L.npts);
      if (L.P && L.Pf) {
        const int ns = p_slots(L.R);
        recast(L.Pf, L.P, (size_t)ns * ns * ns * L.bs * L.cbs * L.npts);
      }
    }
    recast(c.Cpif, c.Cpi, (size_t)11 * c.nF);
    recast(c.pwf, c.pw, c.nF);
  }
}

// The mixed formulation's inner solvers (opt.formulation = 1): the
// displacement hierarchy as for the hybrid form, A_qq as a single face level
// (its Chebyshev smoother stands for the paper's incomplete Cholesky), and
// the smoothed-aggregation hierarchy of C~_p started on the cell lattice.
void build_mixed_hierarchies(Ctx& c) {
  if (c.opt.near_kernel == 1) build_u_rbm(c);
  else build_u(c);
  c.hq.clear();
  Level Q;
  Q.faces = true;
  Q.bs = 1;
  Q.npts = c.nF;
  Q.n = c.nF;
  Q.ell = c.Aqq;
  c.hq.push_back(Q);
  alloc_work(c, c.hq.back());
  finish_level(c, c.hq.back());
  c.hcp.clear();
  Level L0;
  L0.bs = 1;
  L0.A.Lx = c.nx; L0.A.Ly = c.ny; L0.A.Lz = c.nz;
  L0.A.N = c.nT; L0.A.bs = 1; L0.A.kind = ST_DIAMOND2;
  L0.A.val = c.Cp;
  L0.npts = c.nT;
  L0.n = c.nT;
  L0.R = 2;
  L0.active = dalloc_n<unsigned char>(c, c.nT);
  MHFP_CUDA(cudaMemsetAsync(L0.active, 1, c.nT, c.stream));
  c.hcp.push_back(L0);
  while (c.hcp.back().npts > c.opt.coarse_max && c.hcp.size() < 8) {
    Level& L = c.hcp.back();
    alloc_work(c, L);
    finish_level(c, L);
    Level Cl = coarsen(c, L);
    c.hcp.push_back(Cl);
  }
  Level& last = c.hcp.back();
  alloc_work(c, last);
  make_dense_coarse(c, last);
  if (c.opt.autotune)
    for (auto* H : {&c.hu, &c.hcp})
      for (size_t l = 0; l < H->size(); ++l) {
        Level& L = (*H)[l];
        if (L.faces || L.dense_inv || (H == &c.hu && l == 0) || c.opt.schedule) continue;
        autotune_level<double>(c, L);
      }
  if (c.opt.schedule)
    for (auto* H : {&c.hu, &c.hcp})
      for (size_t l = 0; l < H->size(); ++l) {
        Level& L = (*H)[l];
        if (!L.faces && !L.dense_inv && !(H == &c.hu && l == 0)) L.tpp = c.opt.schedule;
      }
}

// x = the Chebyshev smoother of level 0 of H applied to b from x = 0 (the
// mixed formulation's A_qq solve)
void chebyshev_from_zero(Ctx& c, std::vector<Level>& H, const double* b, double* x) {
  smooth<double>(c, H, 0, b, nullptr, x, view(c, H[0], double()).y, false);
}

int level_schedule(Ctx& c, std::vector<Level>& H, int l) {
  const Level& L = H[l];
  if (&H == &c.hu && l == 0) return L.symf ? sym_minb(L) : 0;  // FP64: the full-storage k_cheb_u0
  return L.tpp ? L.tpp : default_schedule(L.A.N, L.bs);
}

// timed as class 4 (displacement) or 5 (interface pressure)
void vcycle(Ctx& c, std::vector<Level>& H, const double* b, double* x) {
  const int cls = (&H == &c.hu) ? 4 : 5;
  timing_begin(c, cls);
  vcycle_level<double>(c, H, 0, b, x);
  timing_end(c, cls, 0.0);
}
void vcycle(Ctx& c, std::vector<Level>& H, const float* b, float* x) {
  const int cls = (&H == &c.hu) ? 4 : 5;
  timing_begin(c, cls);
  vcycle_level<float>(c, H, 0, b, x);
  timing_end(c, cls, 0.0);
}

void level_apply(Ctx& c, std::vector<Level>& H, int l, const double* x, double* y) {
  level_spmv_t<double>(c, H[l], x, nullptr, y);
}

namespace {
__global__ void k_narrow(long long n, const double* __restrict__ x, float* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}
__global__ void k_widen(long long n, const float* __restrict__ x, double* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (double)x[i];
}
}  // namespace

// One V-cycle in the precision of the solve: FP64 directly, or, with
// precision 1, the FP32 cycle on b rounded to FP32 (the FP32 work vectors of
// the whole system, c.tf and c.zf, hold b and x).
void vcycle_api(Ctx& c, std::vector<Level>& H, const double* b, double* x) {
  if (c.opt.precision != 1) {
    vcycle(c, H, b, x);
    return;
  }
  const long long n = H[0].n;
  k_narrow<<<grid_for(n, 256), 256, 0, c.stream>>>(n, b, c.tf);
  MHFP_LAUNCH_CHECK();
  vcycle(c, H, (const float*)c.tf, c.zf);
  k_widen<<<grid_for(n, 256), 256, 0, c.stream>>>(n, c.zf, x);
  MHFP_LAUNCH_CHECK();
}

}  // namespace mhfp
