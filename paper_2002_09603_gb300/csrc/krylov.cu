// Right-preconditioned flexible GMRES(m) (Section 5: GMRES, right
// preconditioning, zero initial guess, stop on the 2-norm of the residual
// relative to the initial one).  Classical Gram-Schmidt applied twice with
// deterministic two-stage reductions; Givens rotations and the triangular
// solve run in one thread on the device; the host reads one 8-byte residual
// estimate per iteration.
#include "common.cuh"

#include <chrono>
#include <cmath>

namespace mhfp {

namespace {

constexpr int RED_BLOCKS = 608;   // 4 x 152 SMs
constexpr int RED_THREADS = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
  __syncthreads();
  return s;  // valid in thread 0
}

// Gram-Schmidt kernels.  On GB300 the FP64 pipe (about 2 FMA per clock per
// SM) bounds these passes, so they are written for occupancy: few registers
// per thread, many rows in flight, independent FMA chains.
constexpr int GS_BLOCKS = 1216;   // 8 x 152 SMs
constexpr int GS_COLS = 8;        // columns per block in the dot kernel (w is read once per 8 columns)
constexpr int GS_DOT_BLOCKS = 608;  // 4 x 152 SMs: about 12 rows per thread, so the
                                    // block reductions' FP64 adds stay small

// partials[c][block] = sum over this block's rows of V[:,c] . w for the
// GS_COLS columns of blockIdx.y; block column 0 also sums w . w into slot
// `ncols` when with_norm.  Skipped entirely when skip && *skip.
// Sum of a[0..7] over the warp by a transposed butterfly: each exchange
// halves the number of live columns per lane, so the eight sums cost 7 + 2
// FP64 adds and shuffles per lane instead of 40.  Lane 4q + r (r = 0..3)
// returns the warp's sum for column q.
__device__ __forceinline__ double warp_sum8(const double (&a)[GS_COLS]) {
  const unsigned lane = threadIdx.x & 31u;
  const bool h16 = lane & 16u, h8 = lane & 8u, h4 = lane & 4u;
  double k[4], m[2];
#pragma unroll
  for (int q = 0; q < 4; ++q)  // columns 4 h16 + q
    k[q] = (h16 ? a[4 + q] : a[q]) + __shfl_xor_sync(0xffffffffu, h16 ? a[q] : a[4 + q], 16);
#pragma unroll
  for (int q = 0; q < 2; ++q)  // columns 4 h16 + 2 h8 + q
    m[q] = (h8 ? k[2 + q] : k[q]) + __shfl_xor_sync(0xffffffffu, h8 ? k[q] : k[2 + q], 8);
  double t = (h4 ? m[1] : m[0]) + __shfl_xor_sync(0xffffffffu, h4 ? m[0] : m[1], 4);  // column lane >> 2
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

// acc[q] += V[:, c0 + q] . w over this thread's rows for q < NC (the
// valid columns of the block's group, so no predicated-off FMA is issued),
// and nw += w . w when NORM
template <int NC, bool NORM>
__device__ __forceinline__ void gs_rows(long long n, const double* __restrict__ V, int c0,
                                        const double* __restrict__ w, double (&acc)[GS_COLS], double& nw) {
  const long long stride = (long long)gridDim.x * blockDim.x;
#pragma unroll 1
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    const double wr = w[r];
#pragma unroll
    for (int q = 0; q < NC; ++q) acc[q] = fma(V[(long long)(c0 + q) * n + r], wr, acc[q]);
    if (NORM) nw = fma(wr, wr, nw);
  }
}

__global__ void __launch_bounds__(RED_THREADS, 4) k_gs_dots(long long n, const double* __restrict__ V, int ncols,
                                                             const double* __restrict__ w,
                                                             double* __restrict__ partials,
                                                             const int* __restrict__ skip, int with_norm,
                                                             long long lb) {
  static_assert(GS_COLS == 8, "warp_sum8 reduces eight columns");
  V = lane_ptr(V, lb);
  w = lane_ptr(w, lb);
  partials = lane_ptr(partials, lb);
  skip = lane_ptr(skip, lb);
  if (skip && *skip) return;
  __shared__ double sh[RED_THREADS / 32][GS_COLS];
  __shared__ double shn[RED_THREADS / 32];
  const int c0 = blockIdx.y * GS_COLS;
  const bool do_norm = with_norm && blockIdx.y == 0;
  double acc[GS_COLS] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, nw = 0.0;
  // block-uniform branch on the number of valid columns in this group
  switch ((ncols - c0 < GS_COLS ? ncols - c0 : GS_COLS) + (do_norm ? 16 : 0)) {
    case 1: gs_rows<1, false>(n, V, c0, w, acc, nw); break;
    case 2: gs_rows<2, false>(n, V, c0, w, acc, nw); break;
    case 3: gs_rows<3, false>(n, V, c0, w, acc, nw); break;
    case 4: gs_rows<4, false>(n, V, c0, w, acc, nw); break;
    case 5: gs_rows<5, false>(n, V, c0, w, acc, nw); break;
    case 6: gs_rows<6, false>(n, V, c0, w, acc, nw); break;
    case 7: gs_rows<7, false>(n, V, c0, w, acc, nw); break;
    case 8: gs_rows<8, false>(n, V, c0, w, acc, nw); break;
    case 17: gs_rows<1, true>(n, V, c0, w, acc, nw); break;
    case 18: gs_rows<2, true>(n, V, c0, w, acc, nw); break;
    case 19: gs_rows<3, true>(n, V, c0, w, acc, nw); break;
    case 20: gs_rows<4, true>(n, V, c0, w, acc, nw); break;
    case 21: gs_rows<5, true>(n, V, c0, w, acc, nw); break;
    case 22: gs_rows<6, true>(n, V, c0, w, acc, nw); break;
    case 23: gs_rows<7, true>(n, V, c0, w, acc, nw); break;
    case 24: gs_rows<8, true>(n, V, c0, w, acc, nw); break;
    default: break;
  }
  const unsigned lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
  const double t = warp_sum8(acc);
  if ((lane & 3u) == 0) sh[wid][lane >> 2] = t;
  if (do_norm) {
    for (int o = 16; o > 0; o >>= 1) nw += __shfl_xor_sync(0xffffffffu, nw, o);
    if (lane == 0) shn[wid] = nw;
  }
  __syncthreads();
  if (threadIdx.x < GS_COLS && c0 + (int)threadIdx.x < ncols) {
    double s = 0.0;
    for (int k = 0; k < RED_THREADS / 32; ++k) s += sh[k][threadIdx.x];
    partials[(long long)(c0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
  }
  if (do_norm && threadIdx.x == 32) {
    double s = 0.0;
    for (int k = 0; k < RED_THREADS / 32; ++k) s += shn[k];
    partials[(long long)ncols * gridDim.x + blockIdx.x] = s;
  }
}

// same reduction, skipped when *skip != 0
__global__ void k_reduce_partials_flag(int nb, const double* __restrict__ partials, double* __restrict__ out,
                                       const int* __restrict__ skip, long long lb);


// out[col] (+)= sum_b partials[col * nb + b] in a fixed order
// the ncols dot products into hout[0..ncols) and, when nrm2 is given, the
// norm partials (row ncols) into *nrm2; same fixed-order sums as below
__global__ void k_reduce_dots(int nb, const double* __restrict__ partials, double* __restrict__ hout, int ncols,
                              double* __restrict__ nrm2, long long lb) {
  partials = lane_ptr(partials, lb);
  hout = lane_ptr(hout, lb);
  nrm2 = lane_ptr(nrm2, lb);
  __shared__ double sh[RED_THREADS / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partials[(long long)blockIdx.x * nb + b];
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) {
    if ((int)blockIdx.x < ncols) hout[blockIdx.x] = s;
    else *nrm2 = s;
  }
}

__global__ void k_reduce_partials(int nb, const double* __restrict__ partials, double* __restrict__ out, int accumulate,
                                  long long lb) {
  partials = lane_ptr(partials, lb);
  out = lane_ptr(out, lb);
  __shared__ double sh[RED_THREADS / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partials[(long long)blockIdx.x * nb + b];
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = accumulate ? out[blockIdx.x] + s : s;
}

__global__ void k_reduce_partials_flag(int nb, const double* __restrict__ partials, double* __restrict__ out,
                                       const int* __restrict__ skip, long long lb) {
  partials = lane_ptr(partials, lb);
  out = lane_ptr(out, lb);
  skip = lane_ptr(skip, lb);
  if (*skip) return;
  __shared__ double sh[RED_THREADS / 32];
  double v = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v += partials[(long long)blockIdx.x * nb + b];
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

// w -= V h as one FMA chain per row, two rows per thread for independent
// chains (ncols + 1 FP64 operations per row, the norm included); partial
// sums of the updated w . w into partials[block] when partials is given
__global__ void __launch_bounds__(RED_THREADS, 8) k_gemv_sub(long long n, const double* __restrict__ V, int ncols,
                                                              const double* __restrict__ h, double* __restrict__ w,
                                                              double* __restrict__ partials,
                                                              const int* __restrict__ skip, long long lb) {
  V = lane_ptr(V, lb);
  h = lane_ptr(h, lb);
  w = lane_ptr(w, lb);
  partials = lane_ptr(partials, lb);
  skip = lane_ptr(skip, lb);
  if (skip && *skip) return;
  __shared__ double sh[RED_THREADS / 32];
  __shared__ double nh[64];
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) nh[c] = -h[c];
  __syncthreads();
  double acc = 0.0;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += 2 * stride) {
    const long long r1 = r + stride;
    const bool two = r1 < n;
    double v0 = w[r], v1 = two ? w[r1] : 0.0;
#pragma unroll 2
    for (int c = 0; c < ncols; ++c) {
      const double* col = V + (long long)c * n;
      v0 = fma(col[r], nh[c], v0);
      if (two) v1 = fma(col[r1], nh[c], v1);
    }
    w[r] = v0;
    acc = fma(v0, v0, acc);
    if (two) {
      w[r1] = v1;
      acc = fma(v1, v1, acc);
    }
  }
  if (partials) {
    const double t = block_sum(acc, sh);
    if (threadIdx.x == 0) partials[blockIdx.x] = t;
  }
}

__global__ void __launch_bounds__(RED_THREADS) k_norm_partials(long long n, const double* __restrict__ x,
                                                                double* __restrict__ partials, long long lb) {
  x = lane_ptr(x, lb);
  partials = lane_ptr(partials, lb);
  __shared__ double sh[RED_THREADS / 32];
  double acc = 0.0;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (long long)gridDim.x * blockDim.x)
    acc += x[r] * x[r];
  const double t = block_sum(acc, sh);
  if (threadIdx.x == 0) partials[blockIdx.x] = t;
}

// x += Z y
// x += Z y with an FP32 Z (every product exact in FP64, the same sums as
// with the widened columns)
__global__ void k_gemv_add_f(long long n, long long ld, const float* __restrict__ Z, int ncols,
                             const double* __restrict__ y, double* __restrict__ x) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = x[r];
  for (int c = 0; c < ncols; ++c) s += (double)Z[(long long)c * ld + r] * y[c];
  x[r] = s;
}

__global__ void k_gemv_add(long long n, const double* __restrict__ Z, int ncols, const double* __restrict__ y,
                           double* __restrict__ x) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  double s = x[r];
  for (int c = 0; c < ncols; ++c) s += Z[(long long)c * n + r] * y[c];
  x[r] = s;
}

__global__ void k_scale_dev(long long n, const double* __restrict__ x, const double* __restrict__ s,
                            double* __restrict__ y, long long lb) {
  x = lane_ptr(x, lb);
  s = lane_ptr(s, lb);
  y = lane_ptr(y, lb);
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) y[r] = x[r] * s[0];
}

__global__ void k_scale_host(long long n, const double* __restrict__ x, double s, double* __restrict__ y) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) y[r] = x[r] * s;
}

// s is a shared elementwise scaling (not a work vector)
__global__ void k_ewise(long long n, const double* __restrict__ x, const double* __restrict__ s, int divide,
                        double* __restrict__ y, long long lb) {
  x = lane_ptr(x, lb);
  y = lane_ptr(y, lb);
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) y[r] = divide ? x[r] / s[r] : x[r] * s[r];
}

// DGKS test (Daniel, Gragg, Kaufman & Stewart, 1976): after one classical
// Gram-Schmidt projection, reorthogonalise only if the norm fell below
// 1/sqrt(2) of its value before the projection.  nrm[0] = ||w||^2 before,
// nrm[1] = ||w||^2 after.  flag = 1 means "skip the second projection";
// when it is skipped h2 is zeroed and the norm after the first pass is
// carried into nrm[2], which the second pass overwrites otherwise.
__global__ void k_dgks(int ncols, const double* __restrict__ nrm, int* __restrict__ flag, double* __restrict__ h2,
                       double* __restrict__ nrm_final, long long lb) {
  nrm = lane_ptr(nrm, lb);
  flag = lane_ptr(flag, lb);
  h2 = lane_ptr(h2, lb);
  nrm_final = lane_ptr(nrm_final, lb);
  const int i = threadIdx.x;
  const bool skip = nrm[1] > 0.5 * nrm[0];
  if (i == 0) {
    *flag = skip ? 1 : 0;
    if (skip) nrm_final[0] = nrm[1];
  }
  if (skip)
    for (int c = i; c < ncols; c += blockDim.x) h2[c] = 0.0;
}

// One Arnoldi step's Hessenberg column: h = h1 + h2 (j+1 entries; h2 null
// after a single Gram-Schmidt pass), the new
// subdiagonal ||w|| = sqrt(nrm2); apply the previous rotations, make the new
// one, update g.  scal[0] = |g_{j+1}|, scal[1] = 1/||w|| (0 on breakdown).
__global__ void k_givens(int j, int m, const double* __restrict__ h1, const double* __restrict__ h2,
                         const double* __restrict__ nrm2, double* __restrict__ H, double* __restrict__ cs,
                         double* __restrict__ sn, double* __restrict__ g, double* __restrict__ scal, long long lb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  h1 = lane_ptr(h1, lb);
  h2 = lane_ptr(h2, lb);
  nrm2 = lane_ptr(nrm2, lb);
  H = lane_ptr(H, lb);
  cs = lane_ptr(cs, lb);
  sn = lane_ptr(sn, lb);
  g = lane_ptr(g, lb);
  scal = lane_ptr(scal, lb);
  double* col = H + (long long)j * (m + 1);
  for (int i = 0; i <= j; ++i) col[i] = h2 ? h1[i] + h2[i] : h1[i];
  const double hn = sqrt(nrm2[0]);
  col[j + 1] = hn;
  for (int i = 0; i < j; ++i) {
    const double t = cs[i] * col[i] + sn[i] * col[i + 1];
    col[i + 1] = -sn[i] * col[i] + cs[i] * col[i + 1];
    col[i] = t;
  }
  const double den = hypot(col[j], col[j + 1]);
  const double c = den > 0.0 ? col[j] / den : 1.0;
  const double s = den > 0.0 ? col[j + 1] / den : 0.0;
  cs[j] = c;
  sn[j] = s;
  col[j] = den;
  col[j + 1] = 0.0;
  g[j + 1] = -s * g[j];
  g[j] = c * g[j];
  scal[0] = fabs(g[j + 1]);
  scal[1] = hn > 0.0 ? 1.0 / hn : 0.0;
}

// back substitution R y = g (k x k upper triangle of the rotated H)
__global__ void k_lsq(int k, int m, const double* __restrict__ H, const double* __restrict__ g, double* __restrict__ y) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s -= H[(long long)c * (m + 1) + i] * y[c];
    const double d = H[(long long)i * (m + 1) + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

__global__ void k_set_g(int m, double beta, double* __restrict__ g) {
  const int i = threadIdx.x + blockIdx.x * blockDim.x;
  if (i <= m) g[i] = (i == 0) ? beta : 0.0;
}


// hout[0..ncols) = V^T w; with nrm2 non-null also ||w||^2 into nrm2[0];
// with skip non-null nothing happens when *skip != 0
void gs_dots(Ctx& c, int ncols, double* hout, double* nrm2, const int* skip) {
  const int wn = nrm2 ? 1 : 0;
  const dim3 grid = lgrid(GS_DOT_BLOCKS, (ncols + GS_COLS - 1) / GS_COLS);
  k_gs_dots<<<grid, RED_THREADS, 0, c.stream>>>(c.n, c.V, ncols, c.w, c.partials, skip, wn, lbytes());
  MHFP_LAUNCH_CHECK();
  if (skip) {
    k_reduce_partials_flag<<<lgrid(ncols), RED_THREADS, 0, c.stream>>>(GS_DOT_BLOCKS, c.partials, hout, skip, lbytes());
  } else {
    k_reduce_dots<<<lgrid(ncols + wn), RED_THREADS, 0, c.stream>>>(GS_DOT_BLOCKS, c.partials, hout, ncols, nrm2, lbytes());
  }
  MHFP_LAUNCH_CHECK();
}

// norm^2 into dst (device)
void norm2_dev(Ctx& c, const double* x, long long n, double* dst) {
  k_norm_partials<<<lgrid(RED_BLOCKS), RED_THREADS, 0, c.stream>>>(n, x, c.partials, lbytes());
  MHFP_LAUNCH_CHECK();
  k_reduce_partials<<<lgrid(1), RED_THREADS, 0, c.stream>>>(RED_BLOCKS, c.partials, dst, 0, lbytes());
  MHFP_LAUNCH_CHECK();
}

double read_scalar(Ctx& c, const double* dsrc) {
  MHFP_CUDA(cudaMemcpyAsync(c.host_scal, dsrc, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  MHFP_CUDA(cudaStreamSynchronize(c.stream));
  return c.host_scal[0];
}

}  // namespace

void ensure_workspace(Ctx& c) {
  const int m = c.opt.restart;
  if (c.m_alloc == m) return;
  if (c.m_alloc != 0) throw Error{MHFP_ERR_STATE, "restart length cannot change after the first solve"};
  c.V = dalloc_n<double>(c, (size_t)(m + 1) * c.n);
  c.w = dalloc_n<double>(c, c.n);
  c.t = dalloc_n<double>(c, c.n);
  c.tmp = dalloc_n<double>(c, c.n);
  c.h = dalloc_n<double>(c, 2 * (size_t)(m + 1));
  c.H = dalloc_n<double>(c, (size_t)(m + 1) * m);
  c.cs = dalloc_n<double>(c, m);
  c.sn = dalloc_n<double>(c, m);
  c.g = dalloc_n<double>(c, m + 1);
  c.yv = dalloc_n<double>(c, m);
  c.npart = GS_BLOCKS;
  c.partials = dalloc_n<double>(c, (size_t)(m + 2) * GS_BLOCKS);
  c.scal = dalloc_n<double>(c, 8);
  c.dflag = dalloc_n<int>(c, 4);
  if (!c.host_scal) MHFP_CUDA(cudaMallocHost(&c.host_scal, 8 * sizeof(double)));
  c.m_alloc = m;
}

// the preconditioned basis Z in the form the set-up asks for (FP32 in the
// mixed-precision solve, FP64 otherwise), allocated on first use
void ensure_zbasis(Ctx& c) {
  ensure_workspace(c);
  const size_t nz = (size_t)c.opt.restart * c.n;
  if (ff_krylov(c)) {
    if (!c.Zf) {
      c.ldz = (c.n + 3) & ~3LL;
      c.Zf = dalloc_n<float>(c, (size_t)c.opt.restart * c.ldz);
    }
  } else if (!c.Z) {
    c.Z = dalloc_n<double>(c, nz);
  }
}

double device_norm2(Ctx& c, const double* x, long long n) {
  ensure_workspace(c);
  norm2_dev(c, x, n, c.scal + 4);
  return std::sqrt(read_scalar(c, c.scal + 4));
}

void vec_scale(Ctx& c, const double* x, const double* s, bool divide, double* y, long long n) {
  k_ewise<<<lgrid(grid_for(n, 256)), 256, 0, c.stream>>>(n, x, s, divide ? 1 : 0, y, lbytes());
  MHFP_LAUNCH_CHECK();
}

// mul is a shared elementwise scaling (not a work vector)
__global__ void k_to_f32(long long n, const double* __restrict__ x, const double* __restrict__ mul,
                         float* __restrict__ y, long long lb) {
  x = lane_ptr(x, lb);
  y = lane_ptr(y, lb);
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) y[r] = (float)(mul ? x[r] * mul[r] : x[r]);
}

__global__ void k_to_f64(long long n, const float* __restrict__ x, double* __restrict__ y) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) y[r] = (double)x[r];
}

// Back substitution with M (Eq. hybridPrec): pi, then p, then u; or, for the
// adjoint, forward substitution with M^T: u, then p, then pi.  The V-cycles
// are symmetric operators (Galerkin levels, R = P^T, the same Chebyshev
// polynomial before and after), so M^T reuses them unchanged.
template <typename T>
void precond_blocks(Ctx& c, const T* t, T* z, T* work_u, T* work_pi, bool transpose) {
  const T* tu = t;
  const T* tp = t + c.nU;
  const T* tpi = tp + c.nT;
  T* zu = z;
  T* zp = z + c.nU;
  T* zpi = zp + c.nT;
  if (!transpose) {
    vcycle(c, c.hpi, tpi, zpi);
    precond_p_step(c, tp, zpi, zp);
    precond_u_rhs(c, tu, zp, work_u);
    vcycle(c, c.hu, (const T*)work_u, zu);
  } else {
    vcycle(c, c.hu, tu, zu);
    precondT_p_step(c, tp, zu, zp);
    precondT_pi_rhs(c, tpi, zp, work_pi);
    vcycle(c, c.hpi, (const T*)work_pi, zpi);
  }
}

// z = M^-1 (v .* mul) (or M^-T) with the FP32 V-cycles and Schur steps; v
// FP64; the FP32 result in zf_out (default: the handle's FP32 work vector)
// and, when z is given, widened into z
void apply_precond_mixed(Ctx& c, const double* v, const double* mul, double* z, bool transpose,
                         float* zf_out = nullptr) {
  const long long n = c.n;
  float* zo = zf_out ? zf_out : c.zf;
  timing_begin(c, 3);
  k_to_f32<<<lgrid(grid_for(n, 256)), 256, 0, c.stream>>>(n, v, mul, c.tf, lbytes());
  MHFP_LAUNCH_CHECK();
  // level-0 right-hand-side buffers are free at the finest levels
  precond_blocks<float>(c, c.tf, zo, c.hu[0].bf, c.hpi[0].bf, transpose);
  if (z) {
    k_to_f64<<<grid_for(n, 256), 256, 0, c.stream>>>(n, zo, z);
    MHFP_LAUNCH_CHECK();
  }
  timing_end(c, 3, 0.0);
}

// M_II^(m) of Eq. (prec) for the mixed formulation [u | p | q], by forward
// substitution: z_u = V_u(v_u), z_q = Chebyshev(A_qq) v_q, then
// z_p = V_Cp(v_p - A_pu z_u - dt A_pq z_q)
void apply_precond_btp(Ctx& c, const double* v, double* z) {
  const double* vu = v;
  const double* vp = v + c.nU;
  const double* vq = vp + c.nT;
  double* zu = z;
  double* zp = z + c.nU;
  double* zq = zp + c.nT;
  timing_begin(c, 3);
  vcycle(c, c.hu, vu, zu);
  chebyshev_from_zero(c, c.hq, vq, zq);
  double* tp = c.hcp[0].b;  // level 0's right-hand-side buffer is free here
  btp_p_rhs(c, vp, zu, zq, tp);
  vcycle(c, c.hcp, (const double*)tp, zp);
  timing_end(c, 3, 0.0);
}

void apply_precond(Ctx& c, const double* v, double* z, bool transpose) {
  if (c.opt.formulation == 1) {
    if (transpose) throw Error{MHFP_ERR_STATE, "the mixed formulation has no transposed preconditioner"};
    apply_precond_btp(c, v, z);
    return;
  }
  if (c.opt.precision == 1) {
    apply_precond_mixed(c, v, nullptr, z, transpose);
    return;
  }
  timing_begin(c, 3);
  precond_blocks<double>(c, v, z, c.hu[0].b, c.hpi[0].b, transpose);
  timing_end(c, 3, 0.0);
}

// Enqueue Arnoldi step j: z_j = M^-1 v_j, w = D_s A z_j, Gram-Schmidt, the
// Givens update, v_{j+1}, and the copy of |g_{j+1}| to pinned host memory.
void enqueue_arnoldi_step(Ctx& c, int j, bool transpose, bool host_copy = true) {
  const int m = c.opt.restart;
  const long long n = c.n;
  double* vj = c.V + (long long)j * n;
  if (ff_krylov(c)) {
    // z_j stays in FP32 (it is the FP32 preconditioner's output): the
    // float-float operator reads it, and x += Z y widens it
    float* zfj = c.Zf + (long long)j * c.ldz;
    apply_precond_mixed(c, vj, c.ds_inv, nullptr, transpose, zfj);  // unscale into the FP32 preconditioner
    apply_operator_arnoldi(c, nullptr, zfj, c.w, c.ds, transpose);  // w = D_s A z_j
  } else {
    double* zj = c.Z + (long long)j * n;
    if (c.opt.precision == 1) {
      apply_precond_mixed(c, vj, c.ds_inv, zj, transpose);  // unscale into the FP32 preconditioner
    } else {
      vec_scale(c, vj, c.ds_inv, false, c.t, n);  // unscale into the preconditioner
      apply_precond(c, c.t, zj, transpose);
    }
    apply_operator_arnoldi(c, zj, c.zf, c.w, c.ds, transpose);  // w = D_s A z_j
  }
  timing_begin(c, 2);
  // classical Gram-Schmidt with the DGKS reorthogonalisation test:
  // h1 = V^T w and ||w||^2; w -= V h1 and ||w||^2; then, only if the
  // norm dropped by more than 1/sqrt(2), h2 = V^T w and w -= V h2
  // (reorth = 0: the first pass alone, the second is not even queued)
  const bool reorth = c.opt.reorth != 0;
  gs_dots(c, j + 1, c.h, c.scal + 4, nullptr);
  k_gemv_sub<<<lgrid(GS_BLOCKS), RED_THREADS, 0, c.stream>>>(n, c.V, j + 1, c.h, c.w, c.partials + (size_t)m * GS_BLOCKS,
                                                     nullptr, lbytes());
  MHFP_LAUNCH_CHECK();
  // one pass: the new norm goes straight to the slot the Givens step reads
  k_reduce_partials<<<lgrid(1), RED_THREADS, 0, c.stream>>>(GS_BLOCKS, c.partials + (size_t)m * GS_BLOCKS,
                                                     reorth ? c.scal + 5 : c.scal + 2, 0, lbytes());
  MHFP_LAUNCH_CHECK();
  if (reorth) {
    k_dgks<<<lgrid(1), 64, 0, c.stream>>>(j + 1, c.scal + 4, c.dflag, c.h + (m + 1), c.scal + 2, lbytes());
    MHFP_LAUNCH_CHECK();
    gs_dots(c, j + 1, c.h + (m + 1), nullptr, c.dflag);
    k_gemv_sub<<<lgrid(GS_BLOCKS), RED_THREADS, 0, c.stream>>>(n, c.V, j + 1, c.h + (m + 1), c.w,
                                                       c.partials + (size_t)m * GS_BLOCKS, c.dflag, lbytes());
    MHFP_LAUNCH_CHECK();
    k_reduce_partials_flag<<<lgrid(1), RED_THREADS, 0, c.stream>>>(GS_BLOCKS, c.partials + (size_t)m * GS_BLOCKS,
                                                           c.scal + 2, c.dflag, lbytes());
    MHFP_LAUNCH_CHECK();
  }
  timing_end(c, 2, 8.0 * n * (2.0 * (j + 1) + 4.0));
  k_givens<<<lgrid(1), 32, 0, c.stream>>>(j, m, c.h, reorth ? c.h + (m + 1) : nullptr, c.scal + 2, c.H, c.cs, c.sn, c.g,
                                   c.scal, lbytes());
  MHFP_LAUNCH_CHECK();
  k_scale_dev<<<lgrid(grid_for(n, 256)), 256, 0, c.stream>>>(n, c.w, c.scal + 1, c.V + (long long)(j + 1) * n, lbytes());
  MHFP_LAUNCH_CHECK();
  if (host_copy) MHFP_CUDA(cudaMemcpyAsync(c.host_scal, c.scal, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
}

namespace {

// Queue Arnoldi step j (no synchronisation).  With graphs enabled the step
// is captured once per (j, transpose) on a private stream and replayed into
// the handle's stream afterwards: one launch instead of about 50.
IterGraph* launch_arnoldi_step(Ctx& c, int j, bool transpose) {
  if (!c.opt.graphs) {
    enqueue_arnoldi_step(c, j, transpose);
    return nullptr;
  }
  auto& G = c.graphs[transpose ? 1 : 0];
  if ((int)G.size() < c.opt.restart) G.resize(c.opt.restart);
  IterGraph& ig = G[j];
  if (!ig.exec) {
    if (!c.cap_stream) MHFP_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
    cudaStream_t user = c.stream;
    const long long l0 = g_launches;
    c.stream = c.cap_stream;
    c.timing.capturing = true;
    c.timing.capture_list = &ig.timed;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      try {
        enqueue_arnoldi_step(c, j, transpose);
      } catch (...) {
        cudaStreamEndCapture(c.cap_stream, &graph);
        if (graph) cudaGraphDestroy(graph);
        c.stream = user;
        c.timing.capturing = false;
        throw;
      }
      e = cudaStreamEndCapture(c.cap_stream, &graph);
    }
    c.stream = user;
    c.timing.capturing = false;
    c.timing.capture_list = nullptr;
    MHFP_CUDA(e);
    ig.nkernels = g_launches - l0;
    g_launches = l0;  // nothing ran during the capture
    e = cudaGraphInstantiate(&ig.exec, graph, 0);
    cudaGraphDestroy(graph);
    MHFP_CUDA(e);
  }
  MHFP_CUDA(cudaGraphLaunch(ig.exec, c.stream));
  g_launches += ig.nkernels;
  return &ig;
}

// queue D_s (b - A x) and its squared norm into host_scal[0]
void enqueue_residual(Ctx& c, const FgState& f) {
  apply_operator(c, f.x, c.tmp, c.ds, f.b, f.transpose);
  norm2_dev(c, c.tmp, c.n, c.scal + 4);
  MHFP_CUDA(cudaMemcpyAsync(c.host_scal, c.scal + 4, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
}

void finish(Ctx& c, FgState& f, double true_rel) {
  f.converged = f.converged || true_rel <= 1.05 * f.tol;
  f.stats.iterations = f.total;
  f.stats.restarts = f.cycles;
  f.stats.converged = f.converged ? 1 : 0;
  f.stats.rel_residual = f.est;
  f.stats.true_rel_residual = true_rel;
  f.stats.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - f.t0).count();
  f.phase = FgState::DONE;
  if (!f.converged) throw Error{MHFP_ERR_NOT_CONVERGED, "FGMRES reached maxit before the tolerance"};
}

}  // namespace

// Start a solve: x = 0 and ||D_s b|| queued; the caller synchronises the
// handle's stream and calls fgmres_advance until the state is DONE.
void fgmres_begin(Ctx& c, FgState& f, const double* b, double* x, double tol, bool transpose) {
  f = FgState{};
  f.b = b;
  f.x = x;
  f.tol = tol;
  f.transpose = transpose;
  f.t0 = std::chrono::steady_clock::now();
  ensure_zbasis(c);
  MHFP_CUDA(cudaMemsetAsync(x, 0, c.n * sizeof(double), c.stream));
  vec_scale(c, b, c.ds, false, c.tmp, c.n);
  norm2_dev(c, c.tmp, c.n, c.scal + 4);
  MHFP_CUDA(cudaMemcpyAsync(c.host_scal, c.scal + 4, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  f.phase = FgState::NEED_BNORM;
}

// One state transition, after the handle's stream has drained: read the
// scalar the last queued work produced and queue the next piece of work.
// Right-preconditioned FGMRES(m), zero initial guess (Section 5), on the
// equilibrated system; a cycle restarts from the true residual, and the
// solve ends when that true residual meets 1.05 tol (or maxit is reached).
void fgmres_advance(Ctx& c, FgState& f) {
  const int m = c.opt.restart;
  const long long n = c.n;
  switch (f.phase) {
    case FgState::NEED_BNORM: {
      f.bnorm = std::sqrt(c.host_scal[0]);
      if (!std::isfinite(f.bnorm)) throw Error{MHFP_ERR_NONFINITE, "non-finite right-hand side"};
      if (f.bnorm == 0.0) {
        f.converged = true;
        f.est = 0.0;
        finish(c, f, 0.0);
        return;
      }
      enqueue_residual(c, f);
      f.phase = FgState::NEED_BETA;
      return;
    }
    case FgState::NEED_BETA: {
      const double beta = std::sqrt(c.host_scal[0]);
      if (!std::isfinite(beta)) throw Error{MHFP_ERR_NONFINITE, "non-finite residual"};
      if (beta <= 1.05 * f.tol * f.bnorm) {
        f.converged = true;
        f.est = beta / f.bnorm;
        finish(c, f, beta / f.bnorm);
        return;
      }
      if (f.total >= c.opt.maxit) {
        finish(c, f, beta / f.bnorm);
        return;
      }
      k_scale_host<<<grid_for(n, 256), 256, 0, c.stream>>>(n, c.tmp, 1.0 / beta, c.V);
      MHFP_LAUNCH_CHECK();
      k_set_g<<<1, 64, 0, c.stream>>>(m, beta, c.g);
      MHFP_LAUNCH_CHECK();
      f.j = 0;
      f.graph = launch_arnoldi_step(c, 0, f.transpose);
      f.phase = FgState::NEED_RESID;
      return;
    }
    case FgState::NEED_RESID: {
      if (f.graph && c.timing.enabled)
        for (auto& t : f.graph->timed) {
          float ms = 0.f;
          MHFP_CUDA(cudaEventElapsedTime(&ms, t.start, t.stop));
          c.timing.total_ms[t.cls] += ms;
          c.timing.launches[t.cls] += 1;
          c.timing.bytes[t.cls] += t.bytes;
        }
      const double resid = c.host_scal[0];
      ++f.total;
      const int k = f.j + 1;
      f.est = resid / f.bnorm;
      if (!std::isfinite(resid)) throw Error{MHFP_ERR_NONFINITE, "non-finite Arnoldi residual"};
      if (resid <= f.tol * f.bnorm || f.total >= c.opt.maxit || k == m) {
        k_lsq<<<1, 32, 0, c.stream>>>(k, m, c.H, c.g, c.yv);
        MHFP_LAUNCH_CHECK();
        if (ff_krylov(c))
          k_gemv_add_f<<<grid_for(n, 256), 256, 0, c.stream>>>(n, c.ldz, c.Zf, k, c.yv, f.x);
        else
          k_gemv_add<<<grid_for(n, 256), 256, 0, c.stream>>>(n, c.Z, k, c.yv, f.x);
        MHFP_LAUNCH_CHECK();
        ++f.cycles;
        enqueue_residual(c, f);
        f.phase = FgState::NEED_BETA;
        return;
      }
      f.j = k;
      f.graph = launch_arnoldi_step(c, f.j, f.transpose);
      return;
    }
    default:
      return;
  }
}

// ---------------------------------------------------------------------------
// Device-driven solve: the whole FGMRES(m) -- restart cycles in a WHILE
// conditional node, Arnoldi step j in IF node j -- is one CUDA graph,
// launched once per solve.  The decisions the host loop makes (stop, restart,
// next step) are taken by single-thread kernels that read the residual
// estimates on the device and set the conditional handles.  Every loop is
// bounded: a cycle runs at most m steps and the WHILE ends once maxit steps
// have run.

// Several lanes (right-hand sides of one handle in lockstep): the control
// kernels run in one thread and walk the lanes, lane l's control block,
// scalars and Hessenberg data lb bytes after lane l - 1's.  A lane whose
// solve has ended (fin) is skipped; the set goes on while any lane has not
// ended, and a cycle's next step opens while any lane is live in it.  With
// one lane every decision is the single solve's.
template <class T>
__device__ __forceinline__ T* lane_at(T* p, int l, long long lb) {
  return (T*)((char*)p + (long long)l * lb);
}

__global__ void k_ctl_init(DevCtl* __restrict__ ctl, const double* __restrict__ nrm2, cudaGraphConditionalHandle hw,
                           int K, long long lb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  bool any = false;
  for (int l = 0; l < K; ++l) {
    DevCtl* c = lane_at(ctl, l, lb);
    const double bn = sqrt(lane_at(nrm2, l, lb)[0]);
    c->bnorm = bn;
    c->tolb = c->tol * bn;
    c->est = 1.0;
    c->true_rel = 0.0;
    c->total = 0;
    c->cycles = 0;
    c->k = 0;
    c->converged = 0;
    c->status = 0;
    c->pad3 = 0;  // cycle starts, a second bound on the WHILE loop
    c->fin = 0;
    c->live = 0;
    if (!isfinite(bn)) {
      c->status = (int)MHFP_ERR_NONFINITE;
      c->fin = 1;
    } else if (bn == 0.0) {
      c->converged = 1;
      c->est = 0.0;
      c->fin = 1;
    } else {
      any = true;
    }
  }
  ctl->decides = 0;
  ctl->steps = 0;
  cudaGraphSetConditional(hw, any ? 1 : 0);
}

// start of a cycle: beta = ||D_s (b - A x)|| per lane; a lane stops, or
// takes part in the cycle; step 0 opens while any lane takes part
__global__ void k_cycle_decide(DevCtl* __restrict__ ctl, const double* __restrict__ nrm2, double* __restrict__ scal,
                               double* __restrict__ g, cudaGraphConditionalHandle hw,
                               const cudaGraphConditionalHandle* __restrict__ hif, int K, long long lb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const int m = ctl->m;
  ctl->decides += 1;
  bool any = false;
  for (int l = 0; l < K; ++l) {
    DevCtl* c = lane_at(ctl, l, lb);
    double* sc = lane_at(scal, l, lb);
    c->k = 0;
    c->live = 0;
    if (c->fin) {
      sc[6] = 0.0;
      continue;
    }
    const double beta = sqrt(lane_at(nrm2, l, lb)[0]);
    c->pad3 += 1;
    // every cycle either runs at least one step (total grows by one) or
    // stops; the count of cycle starts bounds the loop even if a step did
    // not run, so the WHILE node always terminates
    bool stop = c->pad3 > c->maxit + 1;
    if (stop) {
      c->true_rel = beta / c->bnorm;
    } else if (!isfinite(beta)) {
      c->status = (int)MHFP_ERR_NONFINITE;
      stop = true;
    } else if (beta <= 1.05 * c->tolb) {
      c->converged = 1;
      c->est = beta / c->bnorm;
      c->true_rel = beta / c->bnorm;
      stop = true;
    } else if (c->total >= c->maxit) {
      c->true_rel = beta / c->bnorm;
      stop = true;
    }
    if (stop) {
      c->fin = 1;
      sc[6] = 0.0;
      continue;
    }
    c->live = 1;
    any = true;
    double* gl = lane_at(g, l, lb);
    sc[6] = 1.0 / beta;
    gl[0] = beta;
    for (int i = 1; i <= m; ++i) gl[i] = 0.0;
  }
  if (!any) {
    cudaGraphSetConditional(hw, 0);
    for (int j = 0; j < m; ++j) cudaGraphSetConditional(hif[j], 0);
    return;
  }
  cudaGraphSetConditional(hif[0], 1);
  for (int j = 1; j < m; ++j) cudaGraphSetConditional(hif[j], 0);
}

// after Arnoldi step j: count it for every live lane, and open step j+1
// unless no lane is live any more (converged in the Arnoldi estimate, maxit
// or a non-finite residual); a lane that leaves keeps k, its step count of
// this cycle, for the update x += Z y
__global__ void k_step_done(DevCtl* __restrict__ ctl, const double* __restrict__ scal, int j,
                            cudaGraphConditionalHandle hnext, int has_next, cudaGraphConditionalHandle hw, int K,
                            long long lb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl->steps += 1;
  bool any_next = false, all_fin = true;
  for (int l = 0; l < K; ++l) {
    DevCtl* c = lane_at(ctl, l, lb);
    if (c->live) {
      const double resid = lane_at(scal, l, lb)[0];
      c->total += 1;
      c->k = j + 1;
      c->est = resid / c->bnorm;
      bool next = has_next && resid > c->tolb && c->total < c->maxit;
      if (!isfinite(resid)) {
        c->status = (int)MHFP_ERR_NONFINITE;
        c->fin = 1;
        next = false;
      }
      if (!next) c->live = 0;
      any_next = any_next || next;
    }
    all_fin = all_fin && c->fin;
  }
  if (all_fin) cudaGraphSetConditional(hw, 0);
  if (has_next) cudaGraphSetConditional(hnext, any_next ? 1 : 0);
}

__global__ void k_lsq_dev(const DevCtl* __restrict__ ctl, const double* __restrict__ H, const double* __restrict__ g,
                          double* __restrict__ y, long long lb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl = lane_ptr(ctl, lb);
  H = lane_ptr(H, lb);
  g = lane_ptr(g, lb);
  y = lane_ptr(y, lb);
  const int k = ctl->k, m = ctl->m;
  for (int i = k - 1; i >= 0; --i) {
    double s = g[i];
    for (int c = i + 1; c < k; ++c) s -= H[(long long)c * (m + 1) + i] * y[c];
    const double d = H[(long long)i * (m + 1) + i];
    y[i] = d != 0.0 ? s / d : 0.0;
  }
}

template <typename ZT>
__global__ void k_gemv_add_dev(long long n, long long ld, const ZT* __restrict__ Z, const DevCtl* __restrict__ ctl,
                               const double* __restrict__ y, double* __restrict__ x, long long lb) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  Z = lane_ptr(Z, lb);
  ctl = lane_ptr(ctl, lb);
  y = lane_ptr(y, lb);
  x = lane_ptr(x, lb);
  const int k = ctl->k;
  double s = x[r];
  for (int c = 0; c < k; ++c) s += (double)Z[(long long)c * ld + r] * y[c];
  x[r] = s;
}

__global__ void k_cycle_end(DevCtl* __restrict__ ctl, long long lb) {
  ctl = lane_ptr(ctl, lb);
  if (threadIdx.x == 0 && blockIdx.x == 0 && ctl->k > 0) ctl->cycles += 1;
}

namespace {

template <typename... P, typename... A>
cudaGraphNode_t add_kernel(cudaGraph_t g, cudaGraphNode_t dep, void (*f)(P...), dim3 grid, dim3 block, A... args) {
  void* params[] = {(void*)&args...};
  cudaKernelNodeParams kp{};
  kp.func = (void*)f;
  kp.gridDim = grid;
  kp.blockDim = block;
  kp.sharedMemBytes = 0;
  kp.kernelParams = params;
  kp.extra = nullptr;
  cudaGraphNode_t node;
  MHFP_CUDA(cudaGraphAddKernelNode(&node, g, dep ? &dep : nullptr, dep ? 1 : 0, &kp));
  ++g_launches;  // counted like a launch; removed again after the build
  return node;
}

template <class F>
cudaGraph_t capture_piece(Ctx& c, F&& enqueue) {
  if (!c.cap_stream) MHFP_CUDA(cudaStreamCreateWithFlags(&c.cap_stream, cudaStreamNonBlocking));
  cudaStream_t user = c.stream;
  c.stream = c.cap_stream;
  c.suppress_events = true;
  cudaGraph_t graph = nullptr;
  MHFP_CUDA(cudaStreamBeginCapture(c.cap_stream, cudaStreamCaptureModeThreadLocal));
  try {
    enqueue();
  } catch (...) {
    cudaStreamEndCapture(c.cap_stream, &graph);
    if (graph) cudaGraphDestroy(graph);
    c.stream = user;
    c.suppress_events = false;
    throw;
  }
  cudaError_t e = cudaStreamEndCapture(c.cap_stream, &graph);
  c.stream = user;
  c.suppress_events = false;
  MHFP_CUDA(e);
  return graph;
}

cudaGraphNode_t add_child(cudaGraph_t parent, cudaGraphNode_t dep, cudaGraph_t child) {
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphAddChildGraphNode(&node, parent, dep ? &dep : nullptr, dep ? 1 : 0, child);
  cudaGraphDestroy(child);
  MHFP_CUDA(e);
  return node;
}

cudaGraphNode_t add_conditional(cudaGraph_t parent, cudaGraphNode_t dep, cudaGraphConditionalHandle h,
                                cudaGraphConditionalNodeType type, cudaGraph_t* body) {
  cudaGraphNodeParams np{};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  cudaGraphNode_t node;
  MHFP_CUDA(cudaGraphAddNode(&node, parent, dep ? &dep : nullptr, nullptr, dep ? 1 : 0, &np));
  *body = np.conditional.phGraph_out[0];
  return node;
}

__global__ void k_ctl_reset(DevCtl* __restrict__ ctl, double tol, int maxit, int m, long long lb) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  ctl = lane_ptr(ctl, lb);
  DevCtl h{};
  h.tol = tol;
  h.maxit = maxit;
  h.m = m;
  *ctl = h;
}

// Add one whole device-driven solve of handle c to graph G after `dep`:
// [b -> bcur, control block reset] x = 0, ||D_s b||, the control block's
// start, the WHILE node of the restart cycles (Arnoldi steps in IF nodes),
// [xcur -> x] and the control block -> host_slot.  The bracketed parts are
// added when rhs / x are given (batched graphs); the single-solve graph
// leaves them to the host.  d_hif: device array of `restart` IF handles for
// this solve.  With K lanes (c a lane workspace, lane l's work vectors lb
// bytes after lane l - 1's) the solve takes K right-hand sides rhs[0..K)
// in lockstep into x[0..K), control blocks to host_slot[0..K).  Returns the
// last node; the kernel counts go to *cnt.
struct SolveCounts {
  long long start = 0, cycle = 0, step = 0;
};

cudaGraphNode_t add_solve(Ctx& c, cudaGraph_t G, cudaGraphNode_t dep, bool transpose,
                          cudaGraphConditionalHandle* d_hif, const double* const* rhs, double* const* x, double tol,
                          DevCtl* const* host_slot, SolveCounts* cnt, int K = 1, long long lb = 0) {
  const int m = c.opt.restart;
  const long long n = c.n;
  const long long l0 = g_launches;
  LaneScope lanes(K, lb);
  // the WHILE node sits in G, the IF nodes in the WHILE body: each handle is
  // created on the graph that contains its node
  cudaGraphConditionalHandle hw;
  MHFP_CUDA(cudaGraphConditionalHandleCreate(&hw, G, 1, cudaGraphCondAssignDefault));
  DevCtl* ctl = c.ctl;
  cudaGraphNode_t last = dep;
  if (rhs) {
    for (int l = 0; l < K; ++l) {
      cudaGraphNode_t cp;
      MHFP_CUDA(cudaGraphAddMemcpyNode1D(&cp, G, last ? &last : nullptr, last ? 1 : 0,
                                         (char*)c.bcur + (long long)l * lb, rhs[l], n * sizeof(double),
                                         cudaMemcpyDeviceToDevice));
      last = cp;
    }
    last = add_kernel(G, last, k_ctl_reset, lgrid(1), dim3(32), ctl, tol, c.opt.maxit, m, lb);
  }
  // x = 0, ||D_s b|| and the control block
  last = add_child(G, last, capture_piece(c, [&] {
    MHFP_CUDA(lane_memset(c.xcur, 0, n * sizeof(double), c.stream));
    vec_scale(c, c.bcur, c.ds, false, c.tmp, n);
    norm2_dev(c, c.tmp, n, c.scal + 4);
  }));
  last = add_kernel(G, last, k_ctl_init, dim3(1), dim3(32), ctl, (const double*)(c.scal + 4), hw, K, lb);
  const long long nk_start = g_launches - l0;
  cudaGraph_t W;
  cudaGraphNode_t wnode = add_conditional(G, last, hw, cudaGraphCondTypeWhile, &W);
  std::vector<cudaGraphConditionalHandle> hif(m);
  for (int j = 0; j < m; ++j) MHFP_CUDA(cudaGraphConditionalHandleCreate(&hif[j], W, 0, 0));
  MHFP_CUDA(cudaMemcpy(d_hif, hif.data(), m * sizeof(cudaGraphConditionalHandle), cudaMemcpyHostToDevice));
  // while body: the cycle
  const long long l1 = g_launches;
  cudaGraphNode_t b = add_child(W, nullptr, capture_piece(c, [&] {
    apply_operator(c, c.xcur, c.tmp, c.ds, c.bcur, transpose);
    norm2_dev(c, c.tmp, n, c.scal + 4);
  }));
  b = add_kernel(W, b, k_cycle_decide, dim3(1), dim3(32), ctl, (const double*)(c.scal + 4), c.scal, c.g, hw,
                 (const cudaGraphConditionalHandle*)d_hif, K, lb);
  b = add_child(W, b, capture_piece(c, [&] {
    k_scale_dev<<<lgrid(grid_for(n, 256)), 256, 0, c.stream>>>(n, c.tmp, c.scal + 6, c.V, lbytes());
    MHFP_LAUNCH_CHECK();
  }));
  const long long nk_cycle = g_launches - l1;
  long long nk_step = 0;
  for (int j = 0; j < m; ++j) {
    cudaGraph_t body;
    b = add_conditional(W, b, hif[j], cudaGraphCondTypeIf, &body);
    const long long l2 = g_launches;
    cudaGraphNode_t s = add_child(body, nullptr, capture_piece(c, [&] { enqueue_arnoldi_step(c, j, transpose, false); }));
    add_kernel(body, s, k_step_done, dim3(1), dim3(32), ctl, (const double*)c.scal, j,
               j + 1 < m ? hif[j + 1] : hif[j], j + 1 < m ? 1 : 0, hw, K, lb);
    nk_step = g_launches - l2;
  }
  const long long l3 = g_launches;
  b = add_child(W, b, capture_piece(c, [&] {
    k_lsq_dev<<<lgrid(1), 32, 0, c.stream>>>(ctl, c.H, c.g, c.yv, lbytes());
    MHFP_LAUNCH_CHECK();
    if (ff_krylov(c))
      k_gemv_add_dev<float><<<lgrid(grid_for(n, 256)), 256, 0, c.stream>>>(n, c.ldz, c.Zf, ctl, c.yv, c.xcur,
                                                                           lbytes());
    else
      k_gemv_add_dev<double><<<lgrid(grid_for(n, 256)), 256, 0, c.stream>>>(n, n, c.Z, ctl, c.yv, c.xcur,
                                                                            lbytes());
    MHFP_LAUNCH_CHECK();
    k_cycle_end<<<lgrid(1), 32, 0, c.stream>>>(ctl, lbytes());
    MHFP_LAUNCH_CHECK();
  }));
  const long long nk_end = g_launches - l3;
  last = wnode;
  if (x) {
    for (int l = 0; l < K; ++l) {
      cudaGraphNode_t cp;
      MHFP_CUDA(cudaGraphAddMemcpyNode1D(&cp, G, &last, 1, x[l], (const char*)c.xcur + (long long)l * lb,
                                         n * sizeof(double), cudaMemcpyDeviceToDevice));
      last = cp;
    }
  }
  // after the loop: the control blocks back to pinned host memory
  for (int l = 0; l < K; ++l) {
    cudaGraphNode_t fin;
    MHFP_CUDA(cudaGraphAddMemcpyNode1D(&fin, G, &last, 1, host_slot[l], (const char*)ctl + (long long)l * lb,
                                       sizeof(DevCtl), cudaMemcpyDeviceToHost));
    last = fin;
  }
  cnt->start = nk_start;
  cnt->cycle = nk_cycle + nk_end;
  cnt->step = nk_step;
  return last;
}

// the handle's device-side solve state (control block, current b and x)
void ensure_solve_state(Ctx& c) {
  ensure_zbasis(c);
  if (!c.ctl) {
    c.ctl = dalloc_n<DevCtl>(c, 1);
    MHFP_CUDA(cudaMallocHost(&c.host_ctl, sizeof(DevCtl)));
    c.bcur = dalloc_n<double>(c, c.n);
    c.xcur = dalloc_n<double>(c, c.n);
  }
}

void build_solve_graph(Ctx& c, bool transpose) {
  ensure_solve_state(c);
  const int ti = transpose ? 1 : 0;
  if (!c.d_hif[ti]) c.d_hif[ti] = dalloc_n<cudaGraphConditionalHandle>(c, c.opt.restart);
  const long long l0 = g_launches;
  cudaGraph_t G;
  MHFP_CUDA(cudaGraphCreate(&G, 0));
  SolveCounts cnt;
  DevCtl* slot = c.host_ctl;
  try {
    add_solve(c, G, nullptr, transpose, c.d_hif[ti], nullptr, nullptr, 0.0, &slot, &cnt);
  } catch (...) {
    g_launches = l0;
    cudaGraphDestroy(G);
    throw;
  }
  g_launches = l0;  // nothing ran during the build
  cudaGraphExec_t exec;
  cudaError_t e = cudaGraphInstantiate(&exec, G, 0);
  cudaGraphDestroy(G);
  MHFP_CUDA(e);
  c.solve_exec[ti] = exec;
  // launches of one solve = start + per cycle (cycle + end) + per step
  c.solve_nkernels[ti] = cnt.start;
  c.solve_cycle_kernels[ti] = cnt.cycle;
  c.solve_step_kernels[ti] = cnt.step;
}

// A lockstep workspace for K right-hand sides of handle `base`: a copy of
// the handle that shares every matrix, hierarchy and launch schedule, with
// its own work vectors (Krylov basis, Hessenberg data, control block, the
// levels' vectors) carved from one arena: lane 0's at the start, lane l's
// l * lane_bytes further.
Ctx* make_lane_ctx(Ctx& base, int K) {
  if (base.opt.formulation != 0)
    throw Error{MHFP_ERR_STATE, "right-hand sides in lockstep are solved for the hybrid system only"};
  ensure_solve_state(base);
  Ctx* lc = new Ctx(base);
  lc->allocs.clear();
  lc->timing = Timing{};
  lc->suppress_events = false;
  lc->cap_stream = nullptr;
  lc->graphs[0].clear();
  lc->graphs[1].clear();
  lc->solve_exec[0] = lc->solve_exec[1] = nullptr;
  lc->d_hif[0] = lc->d_hif[1] = nullptr;
  lc->host_scal = nullptr;
  lc->host_ctl = nullptr;
  // the lane layout: every work vector at a 256-byte aligned offset
  struct Slot {
    void** p;
    size_t bytes;
  };
  std::vector<Slot> slots;
  const int m = base.opt.restart;
  const size_t n = (size_t)base.n;
  auto add = [&](auto*& p, size_t bytes) { slots.push_back({(void**)&p, bytes}); };
  add(lc->V, (size_t)(m + 1) * n * sizeof(double));
  add(lc->w, n * sizeof(double));
  add(lc->t, n * sizeof(double));
  add(lc->tmp, n * sizeof(double));
  add(lc->h, 2 * (size_t)(m + 1) * sizeof(double));
  add(lc->H, (size_t)(m + 1) * m * sizeof(double));
  add(lc->cs, (size_t)m * sizeof(double));
  add(lc->sn, (size_t)m * sizeof(double));
  add(lc->g, (size_t)(m + 1) * sizeof(double));
  add(lc->yv, (size_t)m * sizeof(double));
  add(lc->partials, (size_t)(m + 2) * GS_BLOCKS * sizeof(double));
  add(lc->scal, 8 * sizeof(double));
  add(lc->dflag, 4 * sizeof(int));
  if (base.Zf) add(lc->Zf, (size_t)m * (size_t)base.ldz * sizeof(float));  // mixed precision: FP32 Z
  if (base.Z) add(lc->Z, (size_t)m * n * sizeof(double));                  // FP64 throughout
  if (base.tf) add(lc->tf, n * sizeof(float));
  if (base.zf) add(lc->zf, n * sizeof(float));
  add(lc->ctl, sizeof(DevCtl));
  add(lc->bcur, n * sizeof(double));
  add(lc->xcur, n * sizeof(double));
  for (auto* H : {&lc->hu, &lc->hpi})
    for (Level& L : *H) {
      const size_t ld = (size_t)L.n * sizeof(double), lf = (size_t)L.n * sizeof(float);
      for (double** v : {&L.x, &L.b, &L.r, &L.d, &L.y})
        if (*v) add(*v, ld);
      for (float** v : {&L.xf, &L.bf, &L.rf, &L.df, &L.yf})
        if (*v) add(*v, lf);
    }
  size_t lane = 0;
  std::vector<size_t> off(slots.size());
  for (size_t i = 0; i < slots.size(); ++i) {
    off[i] = lane;
    lane += (slots[i].bytes + 255) & ~(size_t)255;
  }
  try {
    char* arena = (char*)dalloc(*lc, lane * (size_t)K);
    MHFP_CUDA(cudaMemsetAsync(arena, 0, lane * (size_t)K, base.stream));
    for (size_t i = 0; i < slots.size(); ++i) *slots[i].p = arena + off[i];
    lc->lane_bytes = (long long)lane;
    lc->lanes = K;
  } catch (...) {
    dfree_all(*lc);
    delete lc;
    throw;
  }
  return lc;
}

void destroy_lane_ctx(Ctx* lc) {
  if (!lc) return;
  if (lc->cap_stream) cudaStreamDestroy(lc->cap_stream);
  dfree_all(*lc);
  delete lc;
}

}  // namespace

// One CUDA graph for many solves: every handle's entries run in list order
// in a branch of their own (they share its Krylov workspace); branches of
// different handles are independent, so one launch runs them all.  With
// max_lanes > 1 a handle's entries are taken in sets of up to max_lanes
// right-hand sides, each set one lockstep solve in a workspace of its own.
void build_batch_graph(BatchGraph& B, const std::vector<Ctx*>& cs, const std::vector<const double*>& rhs,
                       const std::vector<double*>& x, double tol, int max_lanes) {
  const long long l0 = g_launches;
  MHFP_CUDA(cudaGraphCreate(&B.graph, 0));
  const int count = (int)cs.size();
  B.counts.assign(count, {0, 0, 0});
  B.lanes.assign(count, 1);
  B.lead.assign(count, 0);
  MHFP_CUDA(cudaMallocHost(&B.host_ctl, (size_t)std::max(count, 1) * sizeof(DevCtl)));
  std::vector<std::pair<Ctx*, cudaGraphNode_t>> tail;  // last node of each handle's branch
  std::vector<bool> taken(count, false);
  try {
    for (int i = 0; i < count; ++i) {
      if (taken[i]) continue;
      Ctx& c = *cs[i];
      // this entry and the next entries of the same handle, up to max_lanes
      std::vector<int> set{i};
      for (int k = i + 1; k < count && (int)set.size() < max_lanes; ++k)
        if (cs[k] == &c && !taken[k]) set.push_back(k);
      for (int e : set) taken[e] = true;
      const int K = (int)set.size();
      ensure_solve_state(c);
      Ctx* run = &c;
      if (K > 1) {
        // one lockstep workspace per (handle, lane count), reused by the
        // handle's later sets, which run after this one in its branch
        Ctx* found = nullptr;
        for (Ctx* lc : B.lane_ctx)
          if (lc->lane_of == &c && lc->lanes == K) found = lc;
        if (!found) {
          found = make_lane_ctx(c, K);
          found->lane_of = &c;
          B.lane_ctx.push_back(found);
        }
        run = found;
      }
      cudaGraphConditionalHandle* d_hif = nullptr;
      MHFP_CUDA(cudaMalloc(&d_hif, (size_t)c.opt.restart * sizeof(cudaGraphConditionalHandle)));
      B.d_hif.push_back(d_hif);
      cudaGraphNode_t dep = nullptr;
      size_t slot = tail.size();
      for (size_t t = 0; t < tail.size(); ++t)
        if (tail[t].first == &c) slot = t;
      if (slot < tail.size()) dep = tail[slot].second;
      std::vector<const double*> r;
      std::vector<double*> xs;
      std::vector<DevCtl*> hs;
      for (int e : set) {
        r.push_back(rhs[e]);
        xs.push_back(x[e]);
        hs.push_back(&B.host_ctl[e]);
        B.lanes[e] = K;
        B.lead[e] = i;
      }
      SolveCounts cnt;
      const cudaGraphNode_t last = add_solve(*run, B.graph, dep, false, d_hif, r.data(), xs.data(), tol, hs.data(),
                                             &cnt, K, K > 1 ? run->lane_bytes : 0);
      B.counts[i] = {cnt.start + 1, cnt.cycle, cnt.step};  // + the control-block reset
      if (slot < tail.size()) tail[slot].second = last;
      else tail.push_back({&c, last});
    }
    g_launches = l0;
    MHFP_CUDA(cudaGraphInstantiate(&B.exec, B.graph, 0));
  } catch (...) {
    g_launches = l0;
    throw;
  }
}

void run_batch_graph(BatchGraph& B, cudaStream_t stream) {
  MHFP_CUDA(cudaGraphLaunch(B.exec, stream));
  MHFP_CUDA(cudaStreamSynchronize(stream));
  for (size_t i = 0; i < B.counts.size(); ++i) {
    if ((int)i != B.lead[i]) continue;  // a set's launches are counted once, at its first entry
    const DevCtl& h = B.host_ctl[i];
    if (B.lanes[i] == 1)
      g_launches += B.counts[i][0] + (long long)(h.cycles + 1) * B.counts[i][1] + (long long)h.total * B.counts[i][2];
    else  // lane 0 counts the set's cycle starts and steps
      g_launches += B.counts[i][0] + (long long)h.decides * B.counts[i][1] + (long long)h.steps * B.counts[i][2];
  }
}

void destroy_batch_graph(BatchGraph& B) {
  if (B.exec) cudaGraphExecDestroy(B.exec);
  if (B.graph) cudaGraphDestroy(B.graph);
  for (auto* p : B.d_hif) cudaFree(p);
  if (B.host_ctl) cudaFreeHost(B.host_ctl);
  for (Ctx* lc : B.lane_ctx) destroy_lane_ctx(lc);
  B = BatchGraph{};
}

void invalidate_graphs(Ctx& c) {
  MHFP_CUDA(cudaStreamSynchronize(c.stream));
  ++c.graph_gen;
  for (int t = 0; t < 2; ++t) {
    for (auto& g : c.graphs[t]) {
      if (g.exec) cudaGraphExecDestroy(g.exec);
      for (auto& p : g.timed) {
        cudaEventDestroy(p.start);
        cudaEventDestroy(p.stop);
      }
    }
    c.graphs[t].clear();
    if (c.solve_exec[t]) cudaGraphExecDestroy(c.solve_exec[t]);
    c.solve_exec[t] = nullptr;
  }
}

void solve_device_graph_launch(Ctx& c, const double* b, double tol, bool transpose) {
  const int t = transpose ? 1 : 0;
  if (!c.solve_exec[t]) build_solve_graph(c, transpose);
  c.solve_t0 = std::chrono::steady_clock::now();
  MHFP_CUDA(cudaMemcpyAsync(c.bcur, b, c.n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  DevCtl h{};
  h.tol = tol;
  h.maxit = c.opt.maxit;
  h.m = c.opt.restart;
  *c.host_ctl = h;
  MHFP_CUDA(cudaMemcpyAsync(c.ctl, c.host_ctl, sizeof(DevCtl), cudaMemcpyHostToDevice, c.stream));
  MHFP_CUDA(cudaGraphLaunch(c.solve_exec[t], c.stream));
  c.solve_pending = t;
}

void solve_device_graph_finish(Ctx& c, double* x, mhfp_stats* st) {
  const int t = c.solve_pending;
  MHFP_CUDA(cudaMemcpyAsync(x, c.xcur, c.n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
  MHFP_CUDA(cudaStreamSynchronize(c.stream));
  const DevCtl& h = *c.host_ctl;
  g_launches += c.solve_nkernels[t] + (long long)(h.cycles + 1) * c.solve_cycle_kernels[t] +
                (long long)h.total * c.solve_step_kernels[t];
  mhfp_stats s{};
  s.iterations = h.total;
  s.restarts = h.cycles;
  s.converged = h.converged;
  s.rel_residual = h.est;
  s.true_rel_residual = h.true_rel;
  s.solve_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - c.solve_t0).count();
  if (st) *st = s;
  if (h.status == (int)MHFP_ERR_NONFINITE) throw Error{MHFP_ERR_NONFINITE, "non-finite value in the solve"};
  if (!h.converged) throw Error{MHFP_ERR_NOT_CONVERGED, "FGMRES reached maxit before the tolerance"};
}

// The bulk-copy sweep records a wait that ran out of time in bit 8 of the
// handle's device flag instead of hanging; read it after a solve.
void check_wait_flag(Ctx& c) {
  if (c.hu.empty() || c.hu[0].tpp != 4 || c.opt.precision != 1) return;
  int h = 0;
  MHFP_CUDA(cudaMemcpyAsync(&h, c.d_flag, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  MHFP_CUDA(cudaStreamSynchronize(c.stream));
  if (h & 8) {
    MHFP_CUDA(cudaMemsetAsync(c.d_flag, 0, sizeof(int), c.stream));
    throw Error{MHFP_ERR_CUDA, "a bulk copy of the finest displacement sweep did not arrive in time"};
  }
}

// Set-up autotuner of the Chebyshev degree (cheb_degree = 0 in the
// options): solve the step's load right-hand side (previous state zero) to
// 1e-8 with degrees 1, 2 and 3, each after one warm-up solve, and keep the
// fastest.  The captured graphs hold the degree's sweeps, so they are
// dropped between candidates and after the choice.
void autotune_cheb_degree(Ctx& c) {
  double* b = dalloc_n<double>(c, c.n);
  double* x = dalloc_n<double>(c, c.n);
  build_rhs(c, nullptr, 1.0, b);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MHFP_CUDA(cudaEventCreate(&e0));
  MHFP_CUDA(cudaEventCreate(&e1));
  int best = 2;
  float best_ms = 1e30f;
  try {
    for (int deg = 1; deg <= 3; ++deg) {
      c.opt.cheb_degree = deg;
      invalidate_graphs(c);
      mhfp_stats st{};
      float ms = 1e30f;
      bool ok = true;
      for (int rep = 0; rep < 2 && ok; ++rep) {
        MHFP_CUDA(cudaEventRecord(e0, c.stream));
        try {
          fgmres_solve(c, b, x, 1e-8, &st);
        } catch (const Error& e) {
          if (e.status != MHFP_ERR_NOT_CONVERGED) throw;
          ok = false;
        }
        MHFP_CUDA(cudaEventRecord(e1, c.stream));
        MHFP_CUDA(cudaEventSynchronize(e1));
        MHFP_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      }
      if (ok && ms < best_ms) {
        best_ms = ms;
        best = deg;
      }
    }
  } catch (...) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c.opt.cheb_degree = best;
  invalidate_graphs(c);
}

void fgmres_solve(Ctx& c, const double* b, double* x, double tol, mhfp_stats* st, bool transpose) {
  if (c.opt.graphs == 2 && !c.timing.enabled) {
    solve_device_graph_launch(c, b, tol, transpose);
    try {
      solve_device_graph_finish(c, x, st);
    } catch (...) {
      check_wait_flag(c);
      throw;
    }
    check_wait_flag(c);
    return;
  }
  FgState f;
  fgmres_begin(c, f, b, x, tol, transpose);
  try {
    while (f.phase != FgState::DONE) {
      MHFP_CUDA(cudaStreamSynchronize(c.stream));
      fgmres_advance(c, f);
    }
  } catch (const Error& e) {
    if (st) *st = f.stats;
    check_wait_flag(c);
    throw;
  }
  if (st) *st = f.stats;
  check_wait_flag(c);
}

}  // namespace mhfp
