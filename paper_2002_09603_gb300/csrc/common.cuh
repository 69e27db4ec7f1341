// Internal declarations shared by the libmhfp translation units.
#pragma once

#include <cuda_runtime.h>

#include <chrono>
#include <cstdint>
#include <string>
#include <array>
#include <vector>

#include "../../include/mhfp.h"

namespace mhfp {
// Node-blocked layout of a finest-level symmetric half (the diagonal 3x3
// block and the 13 blocks of the neighbours after it in stencil order):
// nodes in blocks of 32, each block its 126 rows (slot u, entry e: row
// 9 u + e) of 32 values; value (row, q) at sym_base(q) + 32 row.
__host__ __device__ inline long long sym_base(long long q) { return (q >> 5) * (126 * 32) + (q & 31); }


// ------------------------------------------------------------ error handling
struct Error {
  mhfp_status status;
  std::string msg;
};

#define MHFP_CUDA(call)                                                              \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess)                                                           \
      throw ::mhfp::Error{MHFP_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)}; \
  } while (0)

// every kernel launch of the library is followed by this check, which also
// counts the launch (mhfp_launch_count)
extern long long g_launches;
#define MHFP_LAUNCH_CHECK()         \
  do {                              \
    ++::mhfp::g_launches;           \
    MHFP_CUDA(cudaGetLastError());  \
  } while (0)

inline unsigned grid_for(long long n, int block) {
  long long g = (n + block - 1) / block;
  return (unsigned)(g < 1 ? 1 : g);
}

// ------------------------------------------------------------ lanes
// Several right-hand sides of one handle solved in lockstep ("lanes"): every
// kernel of the solve runs once for all of them, lane l in blockIdx.z.  A
// lane's work vectors sit at the same offset inside its slice of one arena,
// the slices `bytes` apart, so a kernel finds lane l's copy of a work vector
// at p + l * bytes; matrices are shared and never offset.  g_lane is set
// while a lockstep solve is captured into a graph (one host thread captures
// at a time); otherwise it is {1, 0} and every launch is the single-vector
// one.
struct LaneCfg {
  int k = 1;
  long long bytes = 0;
};
extern thread_local LaneCfg g_lane;
inline dim3 lgrid(unsigned x, unsigned y = 1) { return dim3(x, y, (unsigned)g_lane.k); }
inline long long lbytes() { return g_lane.bytes; }
// lane blockIdx.z's copy of work vector p (null stays null)
template <class T>
__device__ __forceinline__ T* lane_ptr(T* p, long long lb) {
  return p ? (T*)((char*)p + (long long)blockIdx.z * lb) : p;
}
template <class T>
__device__ __forceinline__ const T* lane_ptr(const T* p, long long lb) {
  return p ? (const T*)((const char*)p + (long long)blockIdx.z * lb) : p;
}
// lanes for the launches queued while it lives (restores the previous ones)
struct LaneScope {
  LaneCfg saved;
  LaneScope(int k, long long bytes) : saved(g_lane) {
    g_lane.k = k;
    g_lane.bytes = bytes;
  }
  ~LaneScope() { g_lane = saved; }
  LaneScope(const LaneScope&) = delete;
  LaneScope& operator=(const LaneScope&) = delete;
};
// a copy or a fill of a work vector in every lane
inline cudaError_t lane_copy(void* dst, const void* src, size_t bytes, cudaStream_t s) {
  for (int l = 0; l < g_lane.k; ++l) {
    const cudaError_t e = cudaMemcpyAsync((char*)dst + l * g_lane.bytes, (const char*)src + l * g_lane.bytes, bytes,
                                          cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}
inline cudaError_t lane_memset(void* dst, int v, size_t bytes, cudaStream_t s) {
  for (int l = 0; l < g_lane.k; ++l) {
    const cudaError_t e = cudaMemsetAsync((char*)dst + l * g_lane.bytes, v, bytes, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Row blocks that mhfp_residual_norm_noalloc needs for a mesh of nx*ny*nz
// cells: one partial-sum slot per block of 256 rows in each of its three row
// kernels (displacement nodes, cells, faces).  The call accepts a mesh when
// this count is at most the static scratch's 65536 slots (a cube of up to
// about 149^3 cells).  Host-callable so the limit can be checked without a
// GPU.
constexpr long long NOALLOC_ROWS_PER_BLOCK = 256;
constexpr long long NOALLOC_MAX_BLOCKS = 65536;
__host__ __device__ inline long long noalloc_row_blocks(long long nx, long long ny, long long nz) {
  const long long nN = (nx + 1) * (ny + 1) * (nz + 1);
  const long long nT = nx * ny * nz;
  const long long nF = (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1);
  const long long B = NOALLOC_ROWS_PER_BLOCK;
  return (nN + B - 1) / B + (nT + B - 1) / B + (nF + B - 1) / B;
}

// ------------------------------------------------------------ stencils
// Offsets of a structured lattice operator.  BOX1: the 27 neighbours with
// |d|_inf <= 1 (Q1 node coupling), DIAMOND2: the 25 with |d|_1 <= 2 (cell
// coupling through shared faces after faces -> cells), BOX2: the 125 with
// |d|_inf <= 2 (smoothed-aggregation coarse levels of DIAMOND2/BOX2).
enum StencilKind : int { ST_BOX1 = 0, ST_DIAMOND2 = 1, ST_BOX2 = 2 };

__host__ __device__ inline int stencil_size(int k) { return k == ST_BOX1 ? 27 : (k == ST_DIAMOND2 ? 25 : 125); }
__host__ __device__ inline int stencil_radius(int k) { return k == ST_BOX1 ? 1 : 2; }

// offset o of a stencil -> (dx,dy,dz)
__host__ __device__ inline void stencil_offset(int kind, int o, int& dx, int& dy, int& dz) {
  if (kind == ST_BOX1) {
    dx = o % 3 - 1; dy = (o / 3) % 3 - 1; dz = o / 9 - 1;
  } else if (kind == ST_BOX2) {
    dx = o % 5 - 2; dy = (o / 5) % 5 - 2; dz = o / 25 - 2;
  } else {
    // enumerate the |d|_1 <= 2 subset of the 5^3 box in box order
    int c = -1;
    for (int b = 0; b < 125; ++b) {
      int x = b % 5 - 2, y = (b / 5) % 5 - 2, z = b / 25 - 2;
      int l1 = (x < 0 ? -x : x) + (y < 0 ? -y : y) + (z < 0 ? -z : z);
      if (l1 <= 2) {
        ++c;
        if (c == o) { dx = x; dy = y; dz = z; return; }
      }
    }
    dx = dy = dz = 0;
  }
}

// (dx,dy,dz) -> offset index of a stencil, or -1 if not part of it
__host__ __device__ inline int stencil_index(int kind, int dx, int dy, int dz) {
  if (kind == ST_BOX1) {
    if (dx < -1 || dx > 1 || dy < -1 || dy > 1 || dz < -1 || dz > 1) return -1;
    return (dx + 1) + 3 * ((dy + 1) + 3 * (dz + 1));
  }
  if (dx < -2 || dx > 2 || dy < -2 || dy > 2 || dz < -2 || dz > 2) return -1;
  if (kind == ST_BOX2) return (dx + 2) + 5 * ((dy + 2) + 5 * (dz + 2));
  int l1 = (dx < 0 ? -dx : dx) + (dy < 0 ? -dy : dy) + (dz < 0 ? -dz : dz);
  if (l1 > 2) return -1;
  int c = 0;
  int target = (dx + 2) + 5 * ((dy + 2) + 5 * (dz + 2));
  for (int b = 0; b < target; ++b) {
    int x = b % 5 - 2, y = (b / 5) % 5 - 2, z = b / 25 - 2;
    int m = (x < 0 ? -x : x) + (y < 0 ? -y : y) + (z < 0 ? -z : z);
    if (m <= 2) ++c;
  }
  return c;
}

// Structured lattice operator: values stored offset-major, then block entry,
// then lattice point (so a warp of consecutive points reads coalesced).
struct StructOp {
  int Lx = 0, Ly = 0, Lz = 0;
  long long N = 0;
  int bs = 1;
  int kind = ST_BOX1;
  double* val = nullptr;  // [noff][bs*bs][N]
  int noff() const { return stencil_size(kind); }
};

// Per-dimension slot range of smoothed-aggregation prolongators with 3-point
// aggregates along each axis and a fine stencil of radius R:
// fine a lies in the support of coarse J iff 3J - R <= a <= 3J + 2 + R.
__host__ __device__ inline int p_lo(int a, int R) { return (a - R + 6) / 3 - 2; }   // = ceil((a-2-R)/3), a >= 0
__host__ __device__ inline int p_slots(int R) { return (2 + 2 * R) / 3 + 1; }
// Q = A P touches coarse J iff 3J - 2R <= a <= 3J + 2 + 2R.
__host__ __device__ inline int q_lo(int a, int R) { return (a - 2 * R + 6) / 3 - 2; } // = ceil((a-2-2R)/3), a >= 0
__host__ __device__ inline int q_slots(int R) { return (2 + 4 * R) / 3 + 1; }

// q = n / d for every 32-bit n, from a magic multiplier fixed at set-up
struct Div32 {
  unsigned m = 1, d = 1;
  int s1 = 0, s2 = 0;
  static Div32 make(unsigned d) {
    int l = 0;
    while ((1ull << l) < d) ++l;  // l = ceil(log2 d)
    Div32 r;
    r.d = d;
    r.m = (unsigned)(((1ull << 32) * ((1ull << l) - d)) / d + 1);
    r.s1 = l < 1 ? l : 1;
    r.s2 = l < 1 ? 0 : l - 1;
    return r;
  }
  __host__ __device__ __forceinline__ unsigned div(unsigned n) const {
#ifdef __CUDA_ARCH__
    const unsigned t = __umulhi(m, n);
#else
    const unsigned t = (unsigned)(((unsigned long long)m * n) >> 32);
#endif
    return (t + ((n - t) >> s1)) >> s2;
  }
};

// 32-bit face topology with invariant-divisor decoding.  Faces are numbered
// by family: x-faces i + (nx+1)(j + ny k), then y-faces i + nx (j + (ny+1) k),
// then z-faces i + nx (j + ny k); local face 2a (2a+1) of a cell is its face
// on the - (+) side of axis a.
struct FaceTopo32 {
  int nx = 0, ny = 0, nz = 0;
  unsigned nT = 0, nF = 0, nFx = 0, nFy = 0;
  Div32 d_nx1, d_ny, d_nx, d_ny1;
  static FaceTopo32 make(int nx, int ny, int nz, long long nT, long long nF, long long nFx, long long nFy) {
    FaceTopo32 t;
    t.nx = nx; t.ny = ny; t.nz = nz;
    t.nT = (unsigned)nT; t.nF = (unsigned)nF; t.nFx = (unsigned)nFx; t.nFy = (unsigned)nFy;
    t.d_nx1 = Div32::make((unsigned)nx + 1);
    t.d_ny = Div32::make((unsigned)ny);
    t.d_nx = Div32::make((unsigned)nx);
    t.d_ny1 = Div32::make((unsigned)ny + 1);
    return t;
  }
  __host__ __device__ __forceinline__ unsigned cell(int i, int j, int k) const {
    return (unsigned)i + (unsigned)nx * ((unsigned)j + (unsigned)ny * (unsigned)k);
  }
  // face lf (0..5) of cell (i, j, k)
  __host__ __device__ __forceinline__ unsigned face(int i, int j, int k, int lf) const {
    const int ax = lf >> 1, up = lf & 1;
    if (ax == 0) return (unsigned)(i + up) + (unsigned)(nx + 1) * ((unsigned)j + (unsigned)ny * (unsigned)k);
    if (ax == 1) return nFx + (unsigned)i + (unsigned)nx * ((unsigned)(j + up) + (unsigned)(ny + 1) * (unsigned)k);
    return nFx + nFy + (unsigned)i + (unsigned)nx * ((unsigned)j + (unsigned)ny * (unsigned)(k + up));
  }
  // axis of face f and the lattice index (i, j, k) of the cell on its + side
  __host__ __device__ __forceinline__ int decode(unsigned f, int& i, int& j, int& k) const {
    if (f < nFx) {
      const unsigned r = d_nx1.div(f);
      i = (int)(f - r * (unsigned)(nx + 1)); k = (int)d_ny.div(r); j = (int)(r - (unsigned)k * (unsigned)ny);
      return 0;
    }
    if (f < nFx + nFy) {
      const unsigned g = f - nFx, r = d_nx.div(g);
      i = (int)(g - r * (unsigned)nx); k = (int)d_ny1.div(r); j = (int)(r - (unsigned)k * (unsigned)(ny + 1));
      return 1;
    }
    const unsigned g = f - nFx - nFy, r = d_nx.div(g);
    i = (int)(g - r * (unsigned)nx); k = (int)d_ny.div(r); j = (int)(r - (unsigned)k * (unsigned)ny);
    return 2;
  }
  // The up to two cells of face f: slot 0 on the - side (f is its local face
  // 2a+1), slot 1 on the + side (local face 2a); absent cells give ok = false.
  __host__ __device__ __forceinline__ void cells(unsigned f, int c[2][3], bool ok[2], int lf[2]) const {
    int i, j, k;
    const int ax = decode(f, i, j, k);
    c[0][0] = i - (ax == 0); c[0][1] = j - (ax == 1); c[0][2] = k - (ax == 2);
    c[1][0] = i; c[1][1] = j; c[1][2] = k;
    ok[0] = ax == 0 ? i > 0 : (ax == 1 ? j > 0 : k > 0);
    ok[1] = ax == 0 ? i < nx : (ax == 1 ? j < ny : k < nz);
    lf[0] = 2 * ax + 1;
    lf[1] = 2 * ax;
  }
  // The 11 columns of face f's row of the face operators, in the slot order
  // of the stored ELL: 0 = f; 1 + 5 s + q = the q-th local face other than
  // f of cell s (in local-face order); f itself where cell s is absent.
  __host__ __device__ __forceinline__ void ell_cols(unsigned f, unsigned col[11]) const {
    int c[2][3], lf[2];
    bool ok[2];
    cells(f, c, ok, lf);
    col[0] = f;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int q = 0; q < 5; ++q)
        col[1 + 5 * s + q] = ok[s] ? face(c[s][0], c[s][1], c[s][2], q + (q >= lf[s])) : f;
  }
};

// ------------------------------------------------------------ multigrid level
struct Level {
  bool faces = false;         // level 0 of the interface-pressure hierarchy
  long long n = 0;            // unknowns
  long long npts = 0;         // lattice points (or faces)
  int bs = 1;
  StructOp A;                 // lattice operator (unused on the face level)
  double* dinv = nullptr;     // [bs*bs][npts] inverse diagonal blocks
  double lmax = 0.0;
  // prolongator to the next level (lattice levels only): [p_slots^3][bs*bs][npts]
  double* P = nullptr;
  int R = 1;                  // stencil radius of A (L_inf)
  int cbs = 0;                // unknowns per point of the next level (P blocks are bs x cbs)
  const double* ell = nullptr; // face level: its ELL values (null: C~_pi)
  int tpp = 0;                // launch schedule chosen by the autotuner (0: default rule):
                              // 1 = one point per thread, 4/8/16 = warps splitting the
                              // offsets; finest FP32 displacement level: blocks per SM (6, 8)
  unsigned char* active = nullptr;  // [n] free dofs
  // work vectors of length n
  double *x = nullptr, *b = nullptr, *r = nullptr, *d = nullptr, *y = nullptr;
  // last level: dense inverse (n x n, row-major)
  double* dense_inv = nullptr;
  // FP32 copies for the mixed-precision cycle (precision == 1)
  float *valf = nullptr, *dinvf = nullptr, *Pf = nullptr;
  float* symf = nullptr;      // finest displacement level, FP32: symmetric half, node blocks of 32 x 126 rows
  double sweep_us = 0.0;      // autotuner's time of one sweep under the chosen schedule
  float *xf = nullptr, *bf = nullptr, *rf = nullptr, *df = nullptr, *yf = nullptr;
};

// ------------------------------------------------------------ handle
struct TimedPair {
  int cls;
  cudaEvent_t start, stop;
  double bytes;
  bool closed;  // stop recorded (classes nest: M^-1 > V-cycle > sweep)
};

// Timed classes: 0 finest displacement Chebyshev sweeps, 1 operator apply,
// 2 Gram-Schmidt, 3 preconditioner apply M^-1, 4 displacement V-cycle,
// 5 interface-pressure V-cycle
constexpr int TIMING_CLASSES = 7;

// FGMRES control block kept in device memory by the device-driven solve
// (several lanes: one block per lane; fin = the lane's solve has ended,
// live = it takes part in the current cycle's steps; lane 0 also counts the
// set's cycle starts and Arnoldi steps, decides and steps)
struct DevCtl {
  double tol, bnorm, tolb, est, true_rel, pad0, pad1, pad2;
  int maxit, m, total, cycles, k, converged, status, pad3;
  int fin, live, decides, steps;
};

// one captured FGMRES iteration (Arnoldi step j of a cycle)
struct IterGraph {
  cudaGraphExec_t exec = nullptr;
  long long nkernels = 0;
  std::vector<TimedPair> timed;  // event-record nodes inside the graph
};

struct Timing {
  bool enabled = false;
  bool capturing = false;                 // record events as graph nodes
  std::vector<TimedPair>* capture_list = nullptr;
  std::vector<cudaEvent_t> ev_start[TIMING_CLASSES], ev_stop[TIMING_CLASSES];
  size_t used[TIMING_CLASSES] = {};
  long long launches[TIMING_CLASSES] = {};
  double total_ms[TIMING_CLASSES] = {};
  double bytes[TIMING_CLASSES] = {};
};

struct Ctx {
  int device = 0;
  int n_sm = 152;           // multiprocessors of the device
  cudaStream_t stream = nullptr;
  int nx = 0, ny = 0, nz = 0;
  long long nN = 0, nT = 0, nF = 0, nFx = 0, nFy = 0, nU = 0, n = 0;
  double dt = 0;
  double trac[3] = {0, 0, 0};
  mhfp_options opt;
  bool assembled = false, prepared = false;
  std::string err;

  // inputs (device)
  double *coords = nullptr, *E = nullptr, *nu = nullptr, *biot = nullptr, *Seps = nullptr,
         *mu = nullptr, *kappa = nullptr;
  unsigned char *node_fix = nullptr, *face_bc = nullptr;
  int* d_flag = nullptr;  // device error flags

  // assembled blocks (device)
  StructOp Auu;             // ST_BOX1, bs 3, Dirichlet rows/cols zeroed
  double* Aup = nullptr;    // [24][nT], Dirichlet rows zeroed
  double* vol = nullptr;    // [nT]
  double* W = nullptr;      // [36][nT] W_T = A_ww,T^-1
  double* W1 = nullptr;     // [6][nT]  W_T 1
  double* sW = nullptr;     // [nT]     1^T W_T 1
  double* Abar = nullptr;   // [nT]     S_eps|T| + dt 1^T W 1
  double* stabc = nullptr;  // [3][nT]  beta_M|M| to the x/y/z macro partner (0: none)
  double* ApPi = nullptr;   // [6][nT]  A_ppi entries (-W1, 0 on drained faces)
  int* ell_col = nullptr;   // [11][nF]
  double* Apipi = nullptr;  // [11][nF]
  double* Cpi = nullptr;    // [11][nF]
  double* pw = nullptr;     // [nF] faces->cells prolongation weight (0, 1/2, 1)
  double* fu = nullptr;     // [nU] traction load
  double* btilde = nullptr; // [nT]
  double* ds = nullptr;     // [n] equilibration D_s
  double* ds_inv = nullptr; // [n] its inverse (multiplies instead of FP64 divisions)
  double* kappa_ratio = nullptr;  // [3][nT] create-time kappa_q / kappa_0 (permeability updates)
  // persistent scratch of the interface-pressure hierarchy rebuild
  // (permeability updates): Galerkin Q and the Gauss-Jordan workspace
  double* upd_Q = nullptr;
  size_t upd_Q_elems = 0;
  double *gj_A = nullptr, *gj_M = nullptr, *gj_prow = nullptr, *gj_fcol = nullptr;
  int* gj_err = nullptr;
  int gj_n = 0;
  cudaGraphConditionalHandle* d_hif[2] = {nullptr, nullptr};  // IF handles of the solve graphs

  std::vector<Level> hu, hpi;
  // the mixed formulation (opt.formulation = 1), unknowns [u | p | q]
  double* Aqq = nullptr;     // [11][nF] A_qq (ELL, the face operators' slots)
  double* Aqp_c = nullptr;   // [6][nT] A_qp per cell face (-s_lf; 0 on no-flow faces)
  double* Apq_c = nullptr;   // [6][nT] A_pq per cell face (+s_lf; 0 on no-flow faces)
  double* Spp = nullptr;     // [nT] A_pp = S_eps |T|
  double* Cp = nullptr;      // [25][nT] C~_p on the cell lattice (25-point slots)
  std::vector<Level> hq, hcp;  // A_qq's Chebyshev level; C~_p's hierarchy
  // FP32 copies used by the mixed-precision preconditioner
  float *Cpif = nullptr, *pwf = nullptr, *ApPif = nullptr, *btildef = nullptr, *Aupf = nullptr;
  float *tf = nullptr, *zf = nullptr;
  // float-float (hi + lo FP32 pairs) copies for the Arnoldi step's operator
  // in the mixed-precision solve: A_uu's symmetric half in the node-blocked
  // layout (sym_base) and the lo parts of A_up (the hi parts are Aupf)
  float *auu_h = nullptr, *auu_l = nullptr, *aup_l = nullptr;
  // and for its p and pi rows (recomputed after a permeability update): the
  // p block's diagonal Abar + sum of the stabilization coefficients, the
  // stabilization coefficients, A_ppi and A_pipi (ELL), each hi and lo
  float *pd_h = nullptr, *pd_l = nullptr, *st_h = nullptr, *st_l = nullptr, *appi_h = nullptr, *appi_l = nullptr,
        *apipi_h = nullptr, *apipi_l = nullptr;
  double* tmp_pd = nullptr;

  // Krylov workspace
  int m_alloc = 0;
  double *V = nullptr, *Z = nullptr, *w = nullptr, *t = nullptr, *tmp = nullptr;
  float* Zf = nullptr;  // the mixed-precision solve's Z: the preconditioner outputs are FP32 values
  long long ldz = 0;    // its column stride: n rounded up to a multiple of 4 (16-byte aligned columns)
  double *h = nullptr, *H = nullptr, *cs = nullptr, *sn = nullptr, *g = nullptr, *yv = nullptr,
         *partials = nullptr, *scal = nullptr;
  int* dflag = nullptr;  // DGKS decision of the current Arnoldi step
  double* host_scal = nullptr;  // pinned
  int npart = 0;

  Timing timing;
  bool suppress_events = false;  // capture without timing events (conditional bodies)
  std::vector<void*> allocs;
  // CUDA graphs of the Arnoldi steps: [transpose][j]
  cudaStream_t cap_stream = nullptr;
  std::vector<IterGraph> graphs[2];
  // device-driven whole solves (one graph launch per solve): [transpose]
  cudaGraphExec_t solve_exec[2] = {nullptr, nullptr};
  long long solve_nkernels[2] = {0, 0};        // kernels before the cycles
  long long solve_cycle_kernels[2] = {0, 0};  // kernels of one cycle's fixed part
  long long solve_step_kernels[2] = {0, 0};   // kernels of one Arnoldi step
  int solve_pending = 0;
  std::chrono::steady_clock::time_point solve_t0;
  int graph_gen = 0;                     // bumped whenever captured graphs are dropped
  DevCtl* ctl = nullptr;                 // device control block
  DevCtl* host_ctl = nullptr;            // pinned copy
  double *bcur = nullptr, *xcur = nullptr;
  // lockstep workspaces (several right-hand sides of one handle): the
  // handle they belong to, their lane count and the bytes between lanes
  const Ctx* lane_of = nullptr;
  int lanes = 1;
  long long lane_bytes = 0;
};

// resumable FGMRES: each advance consumes one scalar read back from the
// device and queues the next piece of work (used to interleave many handles)
struct FgState {
  enum Phase { NEED_BNORM, NEED_BETA, NEED_RESID, DONE };
  int phase = DONE;
  const double* b = nullptr;
  double* x = nullptr;
  double tol = 0.0;
  bool transpose = false;
  double bnorm = 0.0, est = 1.0;
  int total = 0, cycles = 0, j = 0;
  bool converged = false;
  mhfp_stats stats{};
  std::chrono::steady_clock::time_point t0;
  IterGraph* graph = nullptr;
};

// allocation helpers (tracked, freed at destroy)
void* dalloc(Ctx& c, size_t bytes);
template <class T>
T* dalloc_n(Ctx& c, size_t n) { return (T*)dalloc(c, n * sizeof(T)); }
void dfree_all(Ctx& c);

// timing helpers
int level_schedule(Ctx& c, std::vector<Level>& H, int l);  // effective schedule of a lattice level
void timing_begin(Ctx& c, int cls);
void timing_end(Ctx& c, int cls, double bytes);

// assemble.cu
void assemble_all(Ctx& c);
void build_preconditioner_blocks(Ctx& c);
void build_rhs(Ctx& c, const double* xprev, double scale, double* rhs);
void apply_operator(Ctx& c, const double* x, double* y, const double* scale_out, const double* bsub,
                    bool transpose = false);
// the Arnoldi step's w = D_s A z: with precision = 1 the u rows in float-float
// arithmetic from the FP32 preconditioner output zf (z = zf exactly)
void apply_operator_arnoldi(Ctx& c, const double* z, const float* zf, double* y, const double* scale_out,
                            bool transpose);
void narrow_to_f32(Ctx& c, const double* x, float* y, long long n);  // y = fl32(x)
// the mixed-precision solve: FP32 preconditioner, float-float Arnoldi operator
inline bool ff_krylov(const Ctx& c) { return c.opt.precision == 1 && c.opt.formulation == 0 && c.auu_h != nullptr; }
void precond_p_step(Ctx& c, const double* vp, const double* zpi, double* zp);
void precond_u_rhs(Ctx& c, const double* vu, const double* zp, double* tu);
void precond_p_step(Ctx& c, const float* vp, const float* zpi, float* zp);
void precond_u_rhs(Ctx& c, const float* vu, const float* zp, float* tu);
void make_fp32_blocks(Ctx& c);
void precondT_p_step(Ctx& c, const double* vp, const double* zu, double* zp);
void precondT_p_step(Ctx& c, const float* vp, const float* zu, float* zp);
void precondT_pi_rhs(Ctx& c, const double* vpi, const double* zp, double* tpi);
void precondT_pi_rhs(Ctx& c, const float* vpi, const float* zp, float* tpi);
void grad_logk(Ctx& c, const double* lam, const double* x, double* grad);
void misfit(Ctx& c, const double* x, const double* uzt, const double* pt, double wu, double wp, double* J,
            double* g, double* part, long long npart);
void adjoint_rhs(Ctx& c, const double* g, const double* lam_next, double* rhs);
void ensure_workspace(Ctx& c);
void residual_norm_noalloc(Ctx& c, const double* b, const double* x, double* out);
void update_logk_blocks(Ctx& c, const double* logk);
void build_mixed_blocks(Ctx& c);   // A_qq, A_qp, A_pq, S|T|, C~_p, D_s of the mixed formulation
void apply_operator_mixed(Ctx& c, const double* x, double* y, const double* scale_out, const double* bsub);
void btp_p_rhs(Ctx& c, const double* vp, const double* zu, const double* zq, double* tp);

// amg.cu: the interface-pressure hierarchy and the FP32 copies rebuilt in
// place after a permeability update (same levels, same schedules)
void rebuild_pi_hierarchy(Ctx& c);
// krylov.cu: drop the captured CUDA graphs (their kernel arguments hold the
// old Chebyshev coefficients); the next solve captures them again
void invalidate_graphs(Ctx& c);

// amg.cu
void build_hierarchies(Ctx& c);
void vcycle(Ctx& c, std::vector<Level>& H, const double* b, double* x);
void vcycle(Ctx& c, std::vector<Level>& H, const float* b, float* x);
void level_apply(Ctx& c, std::vector<Level>& H, int l, const double* x, double* y);
void build_mixed_hierarchies(Ctx& c);
void chebyshev_from_zero(Ctx& c, std::vector<Level>& H, const double* b, double* x);
void vcycle_api(Ctx& c, std::vector<Level>& H, const double* b, double* x);  // in the solve's precision

// krylov.cu
// one graph over many solves (mhfp_batch_*)
struct BatchGraph {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  DevCtl* host_ctl = nullptr;                        // pinned, one per entry
  std::vector<cudaGraphConditionalHandle*> d_hif;    // per entry
  std::vector<std::array<long long, 3>> counts;      // kernels: start, per cycle, per step
  std::vector<int> lanes;                            // per entry: lanes of its set (1: a single solve)
  std::vector<int> lead;                             // per entry: the entry holding its set's counters
  std::vector<Ctx*> lane_ctx;                        // owned: lockstep workspaces
};
// max_lanes: entries of one handle are taken, in list order, in sets of at
// most max_lanes right-hand sides solved in lockstep (one launch per kernel
// for the whole set); sets of one handle run one after another
void build_batch_graph(BatchGraph& B, const std::vector<Ctx*>& cs, const std::vector<const double*>& rhs,
                       const std::vector<double*>& x, double tol, int max_lanes = 1);
void run_batch_graph(BatchGraph& B, cudaStream_t stream);
void autotune_cheb_degree(Ctx& c);
void destroy_batch_graph(BatchGraph& B);
void fgmres_solve(Ctx& c, const double* rhs, double* x, double tol, mhfp_stats* st, bool transpose = false);
void fgmres_begin(Ctx& c, FgState& f, const double* b, double* x, double tol, bool transpose);
void fgmres_advance(Ctx& c, FgState& f);
void solve_device_graph_launch(Ctx& c, const double* b, double tol, bool transpose);
void solve_device_graph_finish(Ctx& c, double* x, mhfp_stats* st);
void apply_precond(Ctx& c, const double* v, double* z, bool transpose = false);
double device_norm2(Ctx& c, const double* x, long long n);
void vec_scale(Ctx& c, const double* x, const double* s, bool divide, double* y, long long n);

}  // namespace mhfp
