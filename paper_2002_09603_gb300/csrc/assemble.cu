// Element kernels, static condensation, stabilization, assembly, right-hand
// side and the block operator apply of the hybridized Q1-RT0-P0 system.
//
// Appendix A (element matrices), Eq. (hmfeSys)/(A_33H) (condensation of the
// broken RT0 fluxes), Eq. (J_def)/(stab_A) (macro-element pressure-jump
// stabilization), Section 2.1 (backward-Euler right-hand side).
#include "common.cuh"

#include <cmath>
#include <mutex>

namespace mhfp {

namespace {

constexpr double kGP = 0.57735026918962576451;  // 1/sqrt(3): 2-point Gauss-Legendre

struct Dims {
  int nx, ny, nz;
  long long nN, nT, nF, nFx, nFy;
};

__device__ __forceinline__ long long node_id(const Dims& d, int i, int j, int k) {
  return i + (long long)(d.nx + 1) * (j + (long long)(d.ny + 1) * k);
}
__device__ __forceinline__ long long cell_id(const Dims& d, int i, int j, int k) {
  return i + (long long)d.nx * (j + (long long)d.ny * k);
}
__device__ __forceinline__ long long cell_face(const Dims& d, int i, int j, int k, int lf) {
  switch (lf) {
    case 0: return i + (long long)(d.nx + 1) * (j + (long long)d.ny * k);
    case 1: return (i + 1) + (long long)(d.nx + 1) * (j + (long long)d.ny * k);
    case 2: return d.nFx + i + (long long)d.nx * (j + (long long)(d.ny + 1) * k);
    case 3: return d.nFx + i + (long long)d.nx * ((j + 1) + (long long)(d.ny + 1) * k);
    case 4: return d.nFx + d.nFy + i + (long long)d.nx * (j + (long long)d.ny * k);
    default: return d.nFx + d.nFy + i + (long long)d.nx * (j + (long long)d.ny * (k + 1));
  }
}
// face -> its (up to) two cells: slot 0 = cell on the - side (the face is its
// local face 2*axis+1), slot 1 = cell on the + side (local face 2*axis).
__device__ __forceinline__ void face_cells(const Dims& d, long long f, long long cell[2], int lf[2],
                                           int ijk[2][3]) {
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
  int c[3] = {i, j, k};
  int lim[3] = {d.nx, d.ny, d.nz};
  // minus side
  int cm[3] = {c[0], c[1], c[2]};
  cm[ax] -= 1;
  if (cm[ax] >= 0) {
    cell[0] = cell_id(d, cm[0], cm[1], cm[2]); lf[0] = 2 * ax + 1;
    ijk[0][0] = cm[0]; ijk[0][1] = cm[1]; ijk[0][2] = cm[2];
  } else {
    cell[0] = -1; lf[0] = -1;
  }
  if (c[ax] < lim[ax]) {
    cell[1] = cell_id(d, c[0], c[1], c[2]); lf[1] = 2 * ax;
    ijk[1][0] = c[0]; ijk[1][1] = c[1]; ijk[1][2] = c[2];
  } else {
    cell[1] = -1; lf[1] = -1;
  }
}

__device__ __forceinline__ void q1_ref_grad(int a, double xi, double eta, double zeta, double g[3]) {
  const double sx = (a & 1) ? 1.0 : -1.0, sy = ((a >> 1) & 1) ? 1.0 : -1.0, sz = ((a >> 2) & 1) ? 1.0 : -1.0;
  g[0] = 0.125 * sx * (1.0 + sy * eta) * (1.0 + sz * zeta);
  g[1] = 0.125 * sy * (1.0 + sx * xi) * (1.0 + sz * zeta);
  g[2] = 0.125 * sz * (1.0 + sx * xi) * (1.0 + sy * eta);
}

__device__ __forceinline__ void load_cell_coords(const Dims& d, const double* __restrict__ coords, long long T,
                                                 double X[8][3]) {
  const int i = (int)(T % d.nx), j = (int)((T / d.nx) % d.ny), k = (int)(T / ((long long)d.nx * d.ny));
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const long long n = node_id(d, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
    X[a][0] = coords[3 * n]; X[a][1] = coords[3 * n + 1]; X[a][2] = coords[3 * n + 2];
  }
}

// ---------------------------------------------------------------- K1: Q1
// One warp per cell.  Appendix A: [A_uu]_ab = (grad^s eta_a, C_dr grad^s
// eta_b)_T; for isotropic C_dr the 3x3 block is
//   K_ab(i,j) = int lam d_i N_a d_j N_b + G d_j N_a d_i N_b + G delta_ij grad N_a . grad N_b,
// [A_up]_(a,c) = -b int d_c N_a, |T| = int 1.  2x2x2 Gauss.
constexpr int Q1_WARPS = 4;
__global__ void __launch_bounds__(32 * Q1_WARPS) k_q1(Dims d, const double* __restrict__ coords,
                                                      const double* __restrict__ E, const double* __restrict__ nu,
                                                      const double* __restrict__ biot, double* __restrict__ Ke,
                                                      double* __restrict__ Aup, double* __restrict__ vol,
                                                      int* __restrict__ flag) {
  __shared__ double sG[Q1_WARPS][8][8][3];
  __shared__ double sW[Q1_WARPS][8];
  __shared__ double sX[Q1_WARPS][8][3];
  const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long T = (long long)blockIdx.x * Q1_WARPS + wp;
  if (T >= d.nT) return;  // whole warp leaves together; only __syncwarp below
  const int ci = (int)(T % d.nx), cj = (int)((T / d.nx) % d.ny), ck = (int)(T / ((long long)d.nx * d.ny));
  if (lane < 24) {
    const int a = lane / 3, c = lane % 3;
    sX[wp][a][c] = coords[3 * node_id(d, ci + (a & 1), cj + ((a >> 1) & 1), ck + ((a >> 2) & 1)) + c];
  }
  __syncwarp();
  if (lane < 8) {
    const double xi = (lane & 1) ? kGP : -kGP, eta = ((lane >> 1) & 1) ? kGP : -kGP,
                 zeta = ((lane >> 2) & 1) ? kGP : -kGP;
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    double gr[8][3];
    for (int a = 0; a < 8; ++a) {
      q1_ref_grad(a, xi, eta, zeta, gr[a]);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J[i][j] += sX[wp][a][i] * gr[a][j];
    }
    const double c00 = J[1][1] * J[2][2] - J[1][2] * J[2][1];
    const double c01 = J[1][2] * J[2][0] - J[1][0] * J[2][2];
    const double c02 = J[1][0] * J[2][1] - J[1][1] * J[2][0];
    const double det = J[0][0] * c00 + J[0][1] * c01 + J[0][2] * c02;
    if (!(det > 0.0)) atomicOr(flag, 1);
    const double id = 1.0 / det;
    double Ji[3][3];
    Ji[0][0] = c00 * id; Ji[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) * id; Ji[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) * id;
    Ji[1][0] = c01 * id; Ji[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) * id; Ji[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) * id;
    Ji[2][0] = c02 * id; Ji[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) * id; Ji[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) * id;
    for (int a = 0; a < 8; ++a)
      for (int i = 0; i < 3; ++i)
        sG[wp][lane][a][i] = gr[a][0] * Ji[0][i] + gr[a][1] * Ji[1][i] + gr[a][2] * Ji[2][i];
    sW[wp][lane] = det;  // Gauss weight 1
  }
  __syncwarp();
  const double e = E[T], v = nu[T];
  const double lam = e * v / ((1.0 + v) * (1.0 - 2.0 * v));
  const double G = e / (2.0 * (1.0 + v));
  const long long nT = d.nT;
#pragma unroll 1
  for (int rep = 0; rep < 2; ++rep) {
    const int a = (lane >> 3) + 4 * rep, b = lane & 7;
    double K[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int q = 0; q < 8; ++q) {
      const double w = sW[wp][q];
      const double* ga = sG[wp][q][a];
      const double* gb = sG[wp][q][b];
      const double dot = ga[0] * gb[0] + ga[1] * gb[1] + ga[2] * gb[2];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
          K[i][j] += w * (lam * ga[i] * gb[j] + G * ga[j] * gb[i] + (i == j ? G * dot : 0.0));
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Ke[(long long)((3 * a + i) * 24 + 3 * b + j) * nT + T] = K[i][j];
  }
  if (lane < 24) {
    const int a = lane / 3, c = lane % 3;
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += sW[wp][q] * sG[wp][q][a][c];
    Aup[(long long)lane * nT + T] = -biot[T] * s;
  }
  if (lane == 0) {
    double s = 0.0;
    for (int q = 0; q < 8; ++q) s += sW[wp][q];
    vol[T] = s;
  }
}

// ---------------------------------------------------------------- K2: RT0
// Thread per cell.  [A_ww]_fg = (phi_f, mu kappa^-1 phi_g)_T with the
// contravariant Piola map phi = J phi_hat / det J of the unit-outward-flux
// reference basis (phi_hat of local face 2d / 2d+1 is -(1-xi_d)/8 e_d /
// (1+xi_d)/8 e_d).  Condensation (Eq. hmfeSys): W_T = A_ww,T^-1, W_T 1,
// 1^T W_T 1, Abar_pp,T = S_eps|T| + dt 1^T W_T 1.
__global__ void k_rt0(Dims d, const double* __restrict__ coords, const double* __restrict__ mu,
                      const double* __restrict__ kappa, const double* __restrict__ Seps,
                      const double* __restrict__ vol, double dt, double* __restrict__ Wout,
                      double* __restrict__ W1out, double* __restrict__ sWout, double* __restrict__ Abar,
                      int* __restrict__ flag, double* __restrict__ Aww_out = nullptr) {
  const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= d.nT) return;
  double X[8][3];
  load_cell_coords(d, coords, T, X);
  const double m = mu[T];
  const double kinv[3] = {m / kappa[3 * T], m / kappa[3 * T + 1], m / kappa[3 * T + 2]};
  double A[6][6];
  for (int f = 0; f < 6; ++f)
    for (int g = 0; g < 6; ++g) A[f][g] = 0.0;
  for (int q = 0; q < 8; ++q) {
    const double xq[3] = {(q & 1) ? kGP : -kGP, ((q >> 1) & 1) ? kGP : -kGP, ((q >> 2) & 1) ? kGP : -kGP};
    double J[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    for (int a = 0; a < 8; ++a) {
      double gr[3];
      q1_ref_grad(a, xq[0], xq[1], xq[2], gr);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) J[i][j] += X[a][i] * gr[j];
    }
    const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                       J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                       J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
    if (!(det > 0.0)) atomicOr(flag, 1);
    // M_dd' = sum_i J_id J_id' (mu/kappa_i) / det
    double M[3][3];
    for (int p = 0; p < 3; ++p)
      for (int r = 0; r < 3; ++r) M[p][r] = (J[0][p] * J[0][r] * kinv[0] + J[1][p] * J[1][r] * kinv[1] + J[2][p] * J[2][r] * kinv[2]) / det;
    double val[6];
    for (int f = 0; f < 6; ++f) {
      const int dd = f >> 1;
      val[f] = (f & 1) ? (1.0 + xq[dd]) * 0.125 : -(1.0 - xq[dd]) * 0.125;
    }
    for (int f = 0; f < 6; ++f)
      for (int g = 0; g < 6; ++g) A[f][g] += M[f >> 1][g >> 1] * val[f] * val[g];
  }
  if (Aww_out)
    for (int f = 0; f < 6; ++f)
      for (int g = 0; g < 6; ++g) Aww_out[(long long)(6 * f + g) * d.nT + T] = A[f][g];
  // Cholesky A = L L^T, then W = A^-1 column by column
  double L[6][6];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) L[i][j] = 0.0;
  for (int j = 0; j < 6; ++j) {
    double s = A[j][j];
    for (int k = 0; k < j; ++k) s -= L[j][k] * L[j][k];
    if (!(s > 0.0)) { atomicOr(flag, 2); s = 1e-300; }
    const double ljj = sqrt(s);
    L[j][j] = ljj;
    for (int i = j + 1; i < 6; ++i) {
      double t = A[i][j];
      for (int k = 0; k < j; ++k) t -= L[i][k] * L[j][k];
      L[i][j] = t / ljj;
    }
  }
  double W[6][6];
  for (int c = 0; c < 6; ++c) {
    double y[6];
    for (int i = 0; i < 6; ++i) {
      double t = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) t -= L[i][k] * y[k];
      y[i] = t / L[i][i];
    }
    for (int i = 5; i >= 0; --i) {
      double t = y[i];
      for (int k = i + 1; k < 6; ++k) t -= L[k][i] * W[k][c];
      W[i][c] = t / L[i][i];
    }
  }
  // symmetrise (exact symmetry of the stored inverse)
  double s1 = 0.0;
  for (int f = 0; f < 6; ++f) {
    double r = 0.0;
    for (int g = 0; g < 6; ++g) {
      const double wfg = 0.5 * (W[f][g] + W[g][f]);
      Wout[(long long)(6 * f + g) * d.nT + T] = wfg;
      r += wfg;
    }
    W1out[(long long)f * d.nT + T] = r;
    s1 += r;
  }
  sWout[T] = s1;
  Abar[T] = Seps[T] * vol[T] + dt * s1;
}

// ---------------------------------------------------------------- K3: stab
// Thread per cell.  Eq. (J_def): beta_M |M| on every internal face of the
// macro-element (i>>1, j>>1, k>>1); beta_M = (3b)^2 / [32 (lam + 4G)] with
// volume-averaged lam, G, b over the macro-element's cells.
__global__ void k_stab(Dims d, const double* __restrict__ E, const double* __restrict__ nu,
                       const double* __restrict__ biot, const double* __restrict__ vol,
                       double* __restrict__ stabc) {
  const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= d.nT) return;
  const int i = (int)(T % d.nx), j = (int)((T / d.nx) % d.ny), k = (int)(T / ((long long)d.nx * d.ny));
  const int i0 = i & ~1, j0 = j & ~1, k0 = k & ~1;
  double sv = 0, sl = 0, sg = 0, sb = 0;
  for (int kk = k0; kk < k0 + 2 && kk < d.nz; ++kk)
    for (int jj = j0; jj < j0 + 2 && jj < d.ny; ++jj)
      for (int ii = i0; ii < i0 + 2 && ii < d.nx; ++ii) {
        const long long c = cell_id(d, ii, jj, kk);
        const double e = E[c], v = nu[c], w = vol[c];
        const double lam = e * v / ((1.0 + v) * (1.0 - 2.0 * v));
        const double G = e / (2.0 * (1.0 + v));
        sv += w; sl += lam * w; sg += G * w; sb += biot[c] * w;
      }
  const double lamM = sl / sv, GM = sg / sv, bM = sb / sv;
  const double beta = (3.0 * bM) * (3.0 * bM) / (32.0 * (lamM + 4.0 * GM));
  const double c = beta * sv;
  stabc[T] = ((i ^ 1) < d.nx) ? c : 0.0;
  stabc[d.nT + T] = ((j ^ 1) < d.ny) ? c : 0.0;
  stabc[2 * d.nT + T] = ((k ^ 1) < d.nz) ? c : 0.0;
}

// ---------------------------------------------------------------- K4: A_uu
// Thread per (node, neighbour offset): deterministic gather of the <= 8
// element blocks coupling the two nodes, then the Dirichlet treatment (zero
// row and column of a prescribed component, keep its diagonal).
__global__ void k_assemble_uu(Dims d, const double* __restrict__ Ke, const unsigned char* __restrict__ fix,
                              double* __restrict__ val) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= d.nN * 27) return;
  const int o = (int)(tid / d.nN);
  const long long n = tid - (long long)o * d.nN;
  const int ni = (int)(n % (d.nx + 1)), nj = (int)((n / (d.nx + 1)) % (d.ny + 1)),
            nk = (int)(n / ((long long)(d.nx + 1) * (d.ny + 1)));
  const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
  const int mi = ni + dx, mj = nj + dy, mk = nk + dz;
  double blk[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const bool inside = mi >= 0 && mi <= d.nx && mj >= 0 && mj <= d.ny && mk >= 0 && mk <= d.nz;
  unsigned char fm = 0;
  if (inside) {
    fm = fix[node_id(d, mi, mj, mk)];
    const int zlo = dz == 1 ? nk : nk - 1, zhi = dz == -1 ? nk - 1 : nk;
    const int ylo = dy == 1 ? nj : nj - 1, yhi = dy == -1 ? nj - 1 : nj;
    const int xlo = dx == 1 ? ni : ni - 1, xhi = dx == -1 ? ni - 1 : ni;
    for (int cz = zlo; cz <= zhi; ++cz) {
      if (cz < 0 || cz >= d.nz) continue;
      for (int cy = ylo; cy <= yhi; ++cy) {
        if (cy < 0 || cy >= d.ny) continue;
        for (int cx = xlo; cx <= xhi; ++cx) {
          if (cx < 0 || cx >= d.nx) continue;
          const long long T = cell_id(d, cx, cy, cz);
          const int a = (ni - cx) + 2 * (nj - cy) + 4 * (nk - cz);
          const int b = (mi - cx) + 2 * (mj - cy) + 4 * (mk - cz);
          for (int r = 0; r < 3; ++r)
            for (int s = 0; s < 3; ++s) blk[3 * r + s] += Ke[(long long)((3 * a + r) * 24 + 3 * b + s) * d.nT + T];
        }
      }
    }
  }
  const unsigned char fn = fix[n];
  for (int r = 0; r < 3; ++r)
    for (int s = 0; s < 3; ++s) {
      double v = blk[3 * r + s];
      if (((fn >> r) & 1) || ((fm >> s) & 1)) v = (o == 13 && r == s) ? v : 0.0;
      val[(long long)(o * 9 + 3 * r + s) * d.nN + n] = v;
    }
}

__global__ void k_aup_dirichlet(Dims d, const unsigned char* __restrict__ fix, double* __restrict__ Aup) {
  const long long tid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (tid >= d.nT * 24) return;
  const int e = (int)(tid / d.nT);
  const long long T = tid - (long long)e * d.nT;
  const int a = e / 3, c = e % 3;
  const int i = (int)(T % d.nx), j = (int)((T / d.nx) % d.ny), k = (int)(T / ((long long)d.nx * d.ny));
  const long long n = node_id(d, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
  if ((fix[n] >> c) & 1) Aup[tid] = 0.0;
}

// traction load: thread per node, integral of N_a t over every traction face
// touching the node (2x2 Gauss on the bilinear face).
__global__ void k_face_load(Dims d, const double* __restrict__ coords, const unsigned char* __restrict__ face_bc,
                            const unsigned char* __restrict__ fix, double t0, double t1, double t2,
                            double* __restrict__ fu) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= d.nN) return;
  const int ni = (int)(n % (d.nx + 1)), nj = (int)((n / (d.nx + 1)) % (d.ny + 1)),
            nk = (int)(n / ((long long)(d.nx + 1) * (d.ny + 1)));
  double acc = 0.0;  // integral of N_a over traction faces (times traction later)
  for (int cz = nk - 1; cz <= nk; ++cz) {
    if (cz < 0 || cz >= d.nz) continue;
    for (int cy = nj - 1; cy <= nj; ++cy) {
      if (cy < 0 || cy >= d.ny) continue;
      for (int cx = ni - 1; cx <= ni; ++cx) {
        if (cx < 0 || cx >= d.nx) continue;
        const int a = (ni - cx) + 2 * (nj - cy) + 4 * (nk - cz);
        for (int lf = 0; lf < 6; ++lf) {
          const int ax = lf >> 1, side = lf & 1;
          if (((a >> ax) & 1) != side) continue;
          const long long f = cell_face(d, cx, cy, cz, lf);
          if (!(face_bc[f] & 1)) continue;
          // the two in-face axes, lower first
          const int u = ax == 0 ? 1 : 0, v = ax == 2 ? 1 : 2;
          double Xf[4][3];
          int pos = -1;
          for (int q = 0; q < 4; ++q) {
            int loc = (side << ax) | ((q & 1) << u) | (((q >> 1) & 1) << v);
            if (loc == a) pos = q;
            const long long m = node_id(d, cx + (loc & 1), cy + ((loc >> 1) & 1), cz + ((loc >> 2) & 1));
            Xf[q][0] = coords[3 * m]; Xf[q][1] = coords[3 * m + 1]; Xf[q][2] = coords[3 * m + 2];
          }
          const double ps = (pos & 1) ? 1.0 : -1.0, pt = (pos & 2) ? 1.0 : -1.0;
          for (int gs = 0; gs < 2; ++gs)
            for (int gt = 0; gt < 2; ++gt) {
              const double s = gs ? kGP : -kGP, t = gt ? kGP : -kGP;
              double xs[3] = {0, 0, 0}, xt[3] = {0, 0, 0};
              for (int q = 0; q < 4; ++q) {
                const double qs = (q & 1) ? 1.0 : -1.0, qt = (q & 2) ? 1.0 : -1.0;
                const double dNs = 0.25 * qs * (1.0 + qt * t), dNt = 0.25 * qt * (1.0 + qs * s);
                for (int c = 0; c < 3; ++c) { xs[c] += dNs * Xf[q][c]; xt[c] += dNt * Xf[q][c]; }
              }
              const double cr0 = xs[1] * xt[2] - xs[2] * xt[1], cr1 = xs[2] * xt[0] - xs[0] * xt[2],
                           cr2 = xs[0] * xt[1] - xs[1] * xt[0];
              const double area = sqrt(cr0 * cr0 + cr1 * cr1 + cr2 * cr2);
              acc += area * 0.25 * (1.0 + ps * s) * (1.0 + pt * t);
            }
        }
      }
    }
  }
  const unsigned char fx = fix[n];
  fu[3 * n + 0] = (fx & 1) ? 0.0 : acc * t0;
  fu[3 * n + 1] = (fx & 2) ? 0.0 : acc * t1;
  fu[3 * n + 2] = (fx & 4) ? 0.0 : acc * t2;
}

// ---------------------------------------------------------------- K5
// Thread per cell: B~_p (Eq. app_Bp with the fixed-stress diagonal of the
// M_I^(h) definition) and the masked coupling A_ppi = -W_T 1 (zero on
// drained faces, whose columns are eliminated).
__global__ void k_btilde(Dims d, const double* __restrict__ Auu_diag_src, const double* __restrict__ Aup,
                         const double* __restrict__ Seps, const double* __restrict__ vol,
                         const double* __restrict__ stabc, const double* __restrict__ sW,
                         const double* __restrict__ W1, const unsigned char* __restrict__ face_bc, double dt,
                         double* __restrict__ btilde, double* __restrict__ ApPi) {
  const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= d.nT) return;
  const int i = (int)(T % d.nx), j = (int)((T / d.nx) % d.ny), k = (int)(T / ((long long)d.nx * d.ny));
  double fs = 0.0;
  for (int a = 0; a < 8; ++a) {
    const long long n = node_id(d, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
    for (int c = 0; c < 3; ++c) {
      const double v = Aup[(long long)(3 * a + c) * d.nT + T];
      const double dg = Auu_diag_src[(long long)(13 * 9 + 4 * c) * d.nN + n];
      fs += v * v / dg;
    }
  }
  const double sd = stabc[T] + stabc[d.nT + T] + stabc[2 * d.nT + T];
  btilde[T] = Seps[T] * vol[T] + sd + fs + dt * sW[T];
  for (int lf = 0; lf < 6; ++lf) {
    const long long f = cell_face(d, i, j, k, lf);
    ApPi[(long long)lf * d.nT + T] = (face_bc[f] & 2) ? 0.0 : -W1[(long long)lf * d.nT + T];
  }
}

// Thread per face: ELL rows (11 slots) of A_pipi = sum_T W_T and of
// C~_pi = sum_T [W_T - dt (W_T 1)(W_T 1)^T / B~_T], Dirichlet treatment,
// and the faces -> cells prolongation weight.
__global__ void k_face_ell(Dims d, const double* __restrict__ W, const double* __restrict__ W1,
                           const double* __restrict__ btilde, const unsigned char* __restrict__ face_bc, double dt,
                           int* __restrict__ col, double* __restrict__ Apipi, double* __restrict__ Cpi,
                           double* __restrict__ pw) {
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= d.nF) return;
  long long cell[2];
  int lf[2], ijk[2][3];
  face_cells(d, f, cell, lf, ijk);
  const bool fixed = face_bc[f] & 2;
  double da = 0.0, dc = 0.0;
  const long long nF = d.nF, nT = d.nT;
  for (int s = 0; s < 2; ++s) {
    if (cell[s] < 0) {
      for (int q = 0; q < 5; ++q) {
        col[(1 + 5 * s + q) * nF + f] = (int)f;
        Apipi[(1 + 5 * s + q) * nF + f] = 0.0;
        Cpi[(1 + 5 * s + q) * nF + f] = 0.0;
      }
      continue;
    }
    const long long T = cell[s];
    const int l = lf[s];
    const double w1l = W1[(long long)l * nT + T];
    const double bt = btilde[T];
    const double wll = W[(long long)(6 * l + l) * nT + T];
    da += wll;
    dc += wll - dt * w1l * w1l / bt;
    int q = 0;
    for (int m = 0; m < 6; ++m) {
      if (m == l) continue;
      const long long g = cell_face(d, ijk[s][0], ijk[s][1], ijk[s][2], m);
      const bool gfix = face_bc[g] & 2;
      double va = W[(long long)(6 * l + m) * nT + T];
      double vc = va - dt * w1l * W1[(long long)m * nT + T] / bt;
      if (fixed || gfix) { va = 0.0; vc = 0.0; }
      col[(1 + 5 * s + q) * nF + f] = (int)g;
      Apipi[(1 + 5 * s + q) * nF + f] = va;
      Cpi[(1 + 5 * s + q) * nF + f] = vc;
      ++q;
    }
  }
  col[f] = (int)f;
  Apipi[f] = da;
  Cpi[f] = fixed ? da : dc;
  const int ncell = (cell[0] >= 0) + (cell[1] >= 0);
  pw[f] = fixed ? 0.0 : (ncell == 2 ? 0.5 : 1.0);
}

__global__ void k_scalings(Dims d, const double* __restrict__ Auu, const double* __restrict__ btilde,
                           const double* __restrict__ Cpi, double* __restrict__ ds, double* __restrict__ ds_inv) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nU = 3 * d.nN;
  if (r >= nU + d.nT + d.nF) return;
  double v;
  if (r < nU) {
    const long long n = r / 3;
    const int c = (int)(r % 3);
    v = Auu[(long long)(13 * 9 + 4 * c) * d.nN + n];
  } else if (r < nU + d.nT) {
    v = btilde[r - nU];
  } else {
    v = Cpi[r - nU - d.nT];
  }
  const double sq = sqrt(v);
  ds[r] = 1.0 / sq;
  ds_inv[r] = sq;
}

// ---------------------------------------------------------------- RHS
__global__ void k_rhs(Dims d, const double* __restrict__ fu, const double* __restrict__ Aup,
                      const double* __restrict__ Seps, const double* __restrict__ vol,
                      const double* __restrict__ xprev, double scale, double* __restrict__ b) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nU = 3 * d.nN;
  if (r >= nU + d.nT + d.nF) return;
  if (r < nU) {
    b[r] = scale * fu[r];
  } else if (r < nU + d.nT) {
    const long long T = r - nU;
    double s = 0.0;
    if (xprev) {
      const int i = (int)(T % d.nx), j = (int)((T / d.nx) % d.ny), k = (int)(T / ((long long)d.nx * d.ny));
      for (int a = 0; a < 8; ++a) {
        const long long n = node_id(d, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
        for (int c = 0; c < 3; ++c) s -= Aup[(long long)(3 * a + c) * d.nT + T] * xprev[3 * n + c];
      }
      s += Seps[T] * vol[T] * xprev[nU + T];
    }
    b[r] = s;
  } else {
    b[r] = 0.0;
  }
}

// ---------------------------------------------------------------- operator
// out = so ? so[r] * (bsub ? bsub[r] - y : y) : (bsub ? bsub[r] - y : y)
__device__ __forceinline__ double finish(double y, long long r, const double* so, const double* bsub) {
  double v = bsub ? bsub[r] - y : y;
  return so ? so[r] * v : v;
}

// u rows: A_uu x_u (27-point 3x3-block stencil) + A_up x_p (8 cells).
//
// The transposed operator uses the same kernels: A_H^T = D A_H D^-1 with
// D = diag(I, -I, -dt I) (A_pu = -A_up^T, A_pip = A_ppi^T, A_uu, A_pipi and
// Abar_pp + A_stab symmetric), so A_H^T x only changes the coefficients of
// the off-diagonal blocks: cup (u rows, A_up x_p), cpu and cpi (p rows,
// A_pu x_u and A_ppi x_pi), cpp (pi rows, A_pip x_p).
//
// One thread per (node, component) row: blockDim = (APPLY_U_NODES, 3) with
// threadIdx.y the component, so each warp streams 32 consecutive nodes of one
// coefficient array, every thread carries a single FMA chain (81 + 8 FP64
// FMA), and the 3 x nN threads fill the SMs in one wave of small blocks.
constexpr int APPLY_U_NODES = 64;

__global__ void __launch_bounds__(APPLY_U_NODES * 3) k_apply_u(Dims d, const double* __restrict__ Auu,
                                                              const double* __restrict__ Aup,
                                                              const double* __restrict__ x, double* __restrict__ y,
                                                              const double* __restrict__ so,
                                                              const double* __restrict__ bsub, double cup,
                                                              long long lb) {
  x = lane_ptr(x, lb);
  y = lane_ptr(y, lb);
  bsub = lane_ptr(bsub, lb);
  const long long n = (long long)blockIdx.x * APPLY_U_NODES + threadIdx.x;
  if (n >= d.nN) return;
  const int comp = threadIdx.y;
  const int ni = (int)(n % (d.nx + 1)), nj = (int)((n / (d.nx + 1)) % (d.ny + 1)),
            nk = (int)(n / ((long long)(d.nx + 1) * (d.ny + 1)));
  const long long sy = d.nx + 1, sz = (long long)(d.nx + 1) * (d.ny + 1);
  const long long N = d.nN;
  const double* row = Auu + (long long)(3 * comp) * N + n;  // block entries (comp, 0..2) of offset 0
  double acc = 0.0;
#pragma unroll 3
  for (int dz = -1; dz <= 1; ++dz) {
    const int mk = nk + dz;
    if (mk < 0 || mk > d.nz) continue;
    for (int dy = -1; dy <= 1; ++dy) {
      const int mj = nj + dy;
      if (mj < 0 || mj > d.ny) continue;
      for (int dx = -1; dx <= 1; ++dx) {
        const int mi = ni + dx;
        if (mi < 0 || mi > d.nx) continue;
        const int o = (dx + 1) + 3 * (dy + 1) + 9 * (dz + 1);
        const double* xm = x + 3 * (n + dx + dy * sy + dz * sz);
        const double* v = row + (long long)o * 9 * N;
        acc = fma(v[0], xm[0], acc);
        acc = fma(v[N], xm[1], acc);
        acc = fma(v[2 * N], xm[2], acc);
      }
    }
  }
  const double* xp = x + 3 * N;
  double sp = 0.0;
  for (int cz = nk - 1; cz <= nk; ++cz) {
    if (cz < 0 || cz >= d.nz) continue;
    for (int cy = nj - 1; cy <= nj; ++cy) {
      if (cy < 0 || cy >= d.ny) continue;
      for (int cx = ni - 1; cx <= ni; ++cx) {
        if (cx < 0 || cx >= d.nx) continue;
        const long long T = cell_id(d, cx, cy, cz);
        const int a = (ni - cx) + 2 * (nj - cy) + 4 * (nk - cz);
        sp = fma(Aup[(long long)(3 * a + comp) * d.nT + T], xp[T], sp);
      }
    }
  }
  const long long r = 3 * n + comp;
  y[r] = finish(fma(cup, sp, acc), r, so, bsub);
}

// p rows: A_pu x_u + (Abar_pp + A_stab) x_p + dt A_ppi x_pi.
__global__ void __launch_bounds__(256) k_apply_p(FaceTopo32 t, const double* __restrict__ Aup,
                                                 const double* __restrict__ Abar, const double* __restrict__ stabc,
                                                 const double* __restrict__ ApPi, double cpi,
                                                 const double* __restrict__ x, double* __restrict__ y,
                                                 const double* __restrict__ so, const double* __restrict__ bsub,
                                                 double cpu, long long lb) {
  x = lane_ptr(x, lb);
  y = lane_ptr(y, lb);
  bsub = lane_ptr(bsub, lb);
  // 32-bit cell and node decoding; the same sums in the same order as the
  // definition: A_pu x_u, then the p block, then A_ppi x_pi
  const unsigned T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= t.nT) return;
  const unsigned q = t.d_nx.div(T);
  const int i = (int)(T - q * (unsigned)t.nx), k = (int)t.d_ny.div(q), j = (int)(q - (unsigned)k * (unsigned)t.ny);
  const unsigned Lx = (unsigned)t.nx + 1, Ly = (unsigned)t.ny + 1;
  const unsigned nU = 3 * Lx * Ly * ((unsigned)t.nz + 1);
  double su = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const unsigned n = (unsigned)(i + (a & 1)) + Lx * ((unsigned)(j + ((a >> 1) & 1)) + Ly * (unsigned)(k + (a >> 2)));
#pragma unroll
    for (int c = 0; c < 3; ++c) su -= Aup[(unsigned)(3 * a + c) * t.nT + T] * x[3 * n + c];
  }
  double s = cpu * su;
  const double* xp = x + nU;
  const double cx = stabc[T], cy = stabc[t.nT + T], cz = stabc[2 * t.nT + T];
  double st = (Abar[T] + (cx + cy + cz)) * xp[T];
  if (cx != 0.0) st -= cx * xp[t.cell(i ^ 1, j, k)];
  if (cy != 0.0) st -= cy * xp[t.cell(i, j ^ 1, k)];
  if (cz != 0.0) st -= cz * xp[t.cell(i, j, k ^ 1)];
  s += st;
  const double* xpi = xp + t.nT;
  double c = 0.0;
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) c += ApPi[(unsigned)lf * t.nT + T] * xpi[t.face(i, j, k, lf)];
  s += cpi * c;
  const long long r = (long long)nU + T;
  y[r] = finish(s, r, so, bsub);
}

// pi rows: A_pip x_p + A_pipi x_pi (ELL, 11 slots; the columns follow from
// the face topology, FaceTopo32::ell_cols, in the stored slot order).
__global__ void __launch_bounds__(256) k_apply_pi(FaceTopo32 t, long long nU, const double* __restrict__ ApPi,
                                                  const double* __restrict__ Apipi, const double* __restrict__ x,
                                                  double* __restrict__ y, const double* __restrict__ so,
                                                  const double* __restrict__ bsub, double cpp, long long lb) {
  x = lane_ptr(x, lb);
  y = lane_ptr(y, lb);
  bsub = lane_ptr(bsub, lb);
  const unsigned f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= t.nF) return;
  int c[2][3], lf[2];
  bool ok[2];
  t.cells(f, c, ok, lf);
  const double* xp = x + nU;
  const double* xpi = xp + t.nT;
  double s = 0.0;
  for (int q = 0; q < 2; ++q)
    if (ok[q]) {
      const unsigned T = t.cell(c[q][0], c[q][1], c[q][2]);
      s += ApPi[(long long)lf[q] * t.nT + T] * xp[T];
    }
  s *= cpp;
  unsigned col[11];
  t.ell_cols(f, col);
  double a = 0.0;
#pragma unroll
  for (int q = 0; q < 11; ++q) a += Apipi[(long long)q * t.nF + f] * xpi[col[q]];
  s += a;
  const long long r = nU + t.nT + f;
  y[r] = finish(s, r, so, bsub);
}

// t_p = v_p - A_pu z_u - dt A_pq z_q (A_pu z_u = -sum A_up^T z_u, as in the p
// rows of the operator)
__global__ void __launch_bounds__(256) k_btp_p(FaceTopo32 t, const double* __restrict__ Aup,
                                               const double* __restrict__ Apq, double dt,
                                               const double* __restrict__ vp, const double* __restrict__ zu,
                                               const double* __restrict__ zq, double* __restrict__ tp) {
  const unsigned T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= t.nT) return;
  const unsigned q = t.d_nx.div(T);
  const int i = (int)(T - q * (unsigned)t.nx), k = (int)t.d_ny.div(q), j = (int)(q - (unsigned)k * (unsigned)t.ny);
  const unsigned Lx = (unsigned)t.nx + 1, Ly = (unsigned)t.ny + 1;
  double su = 0.0;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const unsigned n = (unsigned)(i + (a & 1)) + Lx * ((unsigned)(j + ((a >> 1) & 1)) + Ly * (unsigned)(k + (a >> 2)));
#pragma unroll
    for (int c = 0; c < 3; ++c) su -= Aup[(unsigned)(3 * a + c) * t.nT + T] * zu[3 * n + c];
  }
  double cq = 0.0;
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) cq += Apq[(unsigned)lf * t.nT + T] * zq[t.face(i, j, k, lf)];
  tp[T] = vp[T] - su - dt * cq;
}

// ---------------------------------------------------------------- float-float
// <hot:ff_operator> (k_apply_u_ff, k_apply_p_ff, k_apply_pi_ff: the source
// region is hashed so that recorded DRAM counters are dropped once it changes)
// The Arnoldi step's operator rows for u in float-float arithmetic: every
// FP64 coefficient a is held as a_h + a_l (two FP32 values, a_h = fl32(a),
// a_l = fl32(a - a_h): 48 significand bits), every product a z is formed
// exactly by an error-free transformation (TwoProduct with an FMA) and the
// sum is kept as an unevaluated pair (TwoSum, Knuth), the rounding error of
// each step carried in the low word.  z is the FP32 output of the
// preconditioner, so its low word is zero.  The relative error of a row is
// about 2^-44 of the sum of |terms|, against 2^-50 in FP64; FGMRES needs the
// Arnoldi products only to well below its tolerance, and the stopping test
// and restarts use the FP64 operator.  GB300 issues FP32 at about 60x its
// FP64 rate, which moves this kernel off the FP64 pipe.
__device__ __forceinline__ void ff_mac(float& sh, float& sl, float ah, float al, float z) {
  const float pr = __fmul_rn(ah, z);
  float e = __fmaf_rn(ah, z, -pr);  // ah z = pr + e exactly
  e = __fmaf_rn(al, z, e);
  const float t = __fadd_rn(sh, pr);
  const float bp = __fsub_rn(t, sh);
  const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(t, bp)), __fsub_rn(pr, bp));  // sh + pr = t + err exactly
  sh = t;
  sl = __fadd_rn(sl, __fadd_rn(err, e));
}

// y_u = A_uu z_u + cup A_up z_p (then finish: D_s and b as in k_apply_u), one
// thread per node and its three rows; A_uu's symmetric half (hi, lo) in the
// node-blocked layout, the lower blocks read transposed from their owners.
__global__ void __launch_bounds__(256, 4) k_apply_u_ff(Dims d, const float* __restrict__ uh,
                                                       const float* __restrict__ ul, const float* __restrict__ aph,
                                                       const float* __restrict__ apl, const float* __restrict__ z,
                                                       double* __restrict__ y, const double* __restrict__ so,
                                                       const double* __restrict__ bsub, float cup, long long lb) {
  z = lane_ptr(z, lb);
  y = lane_ptr(y, lb);
  bsub = lane_ptr(bsub, lb);
  const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.nN) return;
  const int Lx = d.nx + 1, Ly = d.ny + 1, Lz = d.nz + 1;
  const int i = (int)(p % Lx), j = (int)((p / Lx) % Ly), k = (int)(p / ((long long)Lx * Ly));
  auto in = [&](int a, int b, int c) { return a >= 0 && a < Lx && b >= 0 && b < Ly && c >= 0 && c < Lz; };
  float sh[3] = {0.f, 0.f, 0.f}, sl[3] = {0.f, 0.f, 0.f};
  const long long ob = sym_base(p);
#pragma unroll 1
  for (int u = 0; u <= 13; ++u) {
    const int o = 13 + u, dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
    const long long s = dx + (long long)Lx * (dy + (long long)Ly * dz);
    // both blocks' loads are issued before the pair accumulation (an
    // absent neighbour's loads read the node's own rows and are not used)
    const bool up = in(i + dx, j + dy, k + dz), lo = u > 0 && in(i - dx, j - dy, k - dz);
    const long long qu = up ? p + s : p, ql = lo ? p - s : p;
    const long long qb = sym_base(ql) + u * 9 * 32;
    float oh[9], ol[9], th[9], tl[9], zu[3], zl[3];
#pragma unroll
    for (int e = 0; e < 9; ++e) {
      oh[e] = uh[ob + u * 9 * 32 + e * 32];
      ol[e] = ul[ob + u * 9 * 32 + e * 32];
      th[e] = uh[qb + e * 32];
      tl[e] = ul[qb + e * 32];
    }
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      zu[c] = z[3 * qu + c];
      zl[c] = z[3 * ql + c];
    }
    // own block A(p, p + e_u): row a, column c at entry 3 a + c
    if (up) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        ff_mac(sh[a], sl[a], oh[3 * a], ol[3 * a], zu[0]);
        ff_mac(sh[a], sl[a], oh[3 * a + 1], ol[3 * a + 1], zu[1]);
        ff_mac(sh[a], sl[a], oh[3 * a + 2], ol[3 * a + 2], zu[2]);
      }
    }
    // lower block A(p, p - e_u) = A(p - e_u, p)^T: row a, column c at entry 3 c + a
    if (lo) {
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        ff_mac(sh[a], sl[a], th[a], tl[a], zl[0]);
        ff_mac(sh[a], sl[a], th[3 + a], tl[3 + a], zl[1]);
        ff_mac(sh[a], sl[a], th[6 + a], tl[6 + a], zl[2]);
      }
    }
  }
  // cup A_up z_p over the (up to) eight cells of the node
  const float* zp = z + 3 * d.nN;
  for (int cz = k - 1; cz <= k; ++cz) {
    if (cz < 0 || cz >= d.nz) continue;
    for (int cy = j - 1; cy <= j; ++cy) {
      if (cy < 0 || cy >= d.ny) continue;
      for (int cx = i - 1; cx <= i; ++cx) {
        if (cx < 0 || cx >= d.nx) continue;
        const long long T = cell_id(d, cx, cy, cz);
        const int a = (i - cx) + 2 * (j - cy) + 4 * (k - cz);
        const float zt = cup * zp[T];
#pragma unroll
        for (int comp = 0; comp < 3; ++comp)
          ff_mac(sh[comp], sl[comp], aph[(long long)(3 * a + comp) * d.nT + T], apl[(long long)(3 * a + comp) * d.nT + T],
                 zt);
      }
    }
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const long long r = 3 * p + a;
    y[r] = finish((double)sh[a] + (double)sl[a], r, so, bsub);
  }
}

// p rows in float-float: cpu A_pu z_u + (Abar + A_stab) z_p + cpi A_ppi z_pi,
// each of the three sums carried as a pair and combined in FP64
__global__ void __launch_bounds__(256, 2) k_apply_p_ff(FaceTopo32 t, const float* __restrict__ aph,
                                                    const float* __restrict__ apl, const float* __restrict__ pdh,
                                                    const float* __restrict__ pdl, const float* __restrict__ sth,
                                                    const float* __restrict__ stl, const float* __restrict__ pph,
                                                    const float* __restrict__ ppl, double cpi,
                                                    const float* __restrict__ z, double* __restrict__ y,
                                                    const double* __restrict__ so, double cpu, long long lb) {
  z = lane_ptr(z, lb);
  y = lane_ptr(y, lb);
  const unsigned T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= t.nT) return;
  const unsigned q = t.d_nx.div(T);
  const int i = (int)(T - q * (unsigned)t.nx), k = (int)t.d_ny.div(q), j = (int)(q - (unsigned)k * (unsigned)t.ny);
  const unsigned Lx = (unsigned)t.nx + 1, Ly = (unsigned)t.ny + 1;
  const unsigned nU = 3 * Lx * Ly * ((unsigned)t.nz + 1);
  // every load of the row is issued before the (serial) pair accumulation
  float va[24], vb[24], vz[24];
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const unsigned n = (unsigned)(i + (a & 1)) + Lx * ((unsigned)(j + ((a >> 1) & 1)) + Ly * (unsigned)(k + (a >> 2)));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      va[3 * a + c] = aph[(unsigned)(3 * a + c) * t.nT + T];
      vb[3 * a + c] = apl[(unsigned)(3 * a + c) * t.nT + T];
      vz[3 * a + c] = z[3 * n + c];
    }
  }
  float uh = 0.f, ul = 0.f;  // A_up^T z_u (the row is its negative)
#pragma unroll
  for (int e = 0; e < 24; ++e) ff_mac(uh, ul, va[e], vb[e], vz[e]);
  const float* zp = z + nU;
  float ph = 0.f, pl = 0.f;
  ff_mac(ph, pl, pdh[T], pdl[T], zp[T]);
  const unsigned nb[3] = {t.cell(i ^ 1, j, k), t.cell(i, j ^ 1, k), t.cell(i, j, k ^ 1)};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const float ch = sth[d * t.nT + T];
    if (ch != 0.f) ff_mac(ph, pl, -ch, -stl[d * t.nT + T], zp[nb[d]]);
  }
  const float* zpi = zp + t.nT;
  float wa[6], wb[6], wz[6];
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) {
    wa[lf] = pph[lf * t.nT + T];
    wb[lf] = ppl[lf * t.nT + T];
    wz[lf] = zpi[t.face(i, j, k, lf)];
  }
  float ch = 0.f, cl = 0.f;
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) ff_mac(ch, cl, wa[lf], wb[lf], wz[lf]);
  const double s = -cpu * ((double)uh + (double)ul) + ((double)ph + (double)pl) + cpi * ((double)ch + (double)cl);
  const long long r = (long long)nU + T;
  y[r] = finish(s, r, so, nullptr);
}

// pi rows in float-float: cpp A_pip z_p + A_pipi z_pi (ELL, 11 slots)
__global__ void __launch_bounds__(256, 3) k_apply_pi_ff(FaceTopo32 t, long long nU, const float* __restrict__ pph,
                                                     const float* __restrict__ ppl, const float* __restrict__ eh,
                                                     const float* __restrict__ el, const float* __restrict__ z,
                                                     double* __restrict__ y, const double* __restrict__ so,
                                                     double cpp, long long lb) {
  z = lane_ptr(z, lb);
  y = lane_ptr(y, lb);
  const unsigned f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= t.nF) return;
  int c[2][3], lf[2];
  bool ok[2];
  t.cells(f, c, ok, lf);
  const float* zp = z + nU;
  const float* zpi = zp + t.nT;
  float ph = 0.f, pl = 0.f;
  for (int q = 0; q < 2; ++q)
    if (ok[q]) {
      const unsigned T = t.cell(c[q][0], c[q][1], c[q][2]);
      ff_mac(ph, pl, pph[(long long)lf[q] * t.nT + T], ppl[(long long)lf[q] * t.nT + T], zp[T]);
    }
  unsigned col[11];
  t.ell_cols(f, col);
  float va[11], vb[11], vz[11];  // every load issued before the pair accumulation
#pragma unroll
  for (int q = 0; q < 11; ++q) {
    va[q] = eh[(long long)q * t.nF + f];
    vb[q] = el[(long long)q * t.nF + f];
    vz[q] = zpi[col[q]];
  }
  float ah = 0.f, al = 0.f;
#pragma unroll
  for (int q = 0; q < 11; ++q) ff_mac(ah, al, va[q], vb[q], vz[q]);
  const double s = cpp * ((double)ph + (double)pl) + ((double)ah + (double)al);
  const long long r = nU + t.nT + f;
  y[r] = finish(s, r, so, nullptr);
}

// </hot:ff_operator>

// the p block's diagonal Abar + sum of the three stabilization coefficients
__global__ void k_pdiag(long long nT, const double* __restrict__ Abar, const double* __restrict__ stabc,
                        double* __restrict__ out) {
  const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (T < nT) out[T] = Abar[T] + (stabc[T] + stabc[nT + T] + stabc[2 * nT + T]);
}
__global__ void k_split(long long n, const double* __restrict__ x, float* __restrict__ h, float* __restrict__ l) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const float vh = __double2float_rn(x[t]);
  h[t] = vh;
  l[t] = __double2float_rn(x[t] - (double)vh);
}

// FP64 rows into the node-blocked float-float layout (hi = fl32(v), lo =
// fl32(v - hi)); and the lo words of a block array whose hi words exist
__global__ void k_split_sym(long long n, const double* __restrict__ x, float* __restrict__ h, float* __restrict__ l) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 126 * n) return;
  const long long row = t / n, q = t % n;
  const double v = x[t];
  const float vh = __double2float_rn(v);
  h[sym_base(q) + 32 * row] = vh;
  l[sym_base(q) + 32 * row] = __double2float_rn(v - (double)vh);
}
__global__ void k_split_lo(long long n, const double* __restrict__ x, const float* __restrict__ h,
                           float* __restrict__ l) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) l[t] = __double2float_rn(x[t] - (double)h[t]);
}

// preconditioner pieces: z_p = B~^-1 (v_p - dt A_ppi z_pi), t_u = v_u - A_up z_p
// (FP64, or FP32 in the mixed-precision preconditioner)
template <typename R>
__global__ void __launch_bounds__(256) k_prec_p(FaceTopo32 t, const R* __restrict__ ApPi,
                                                const R* __restrict__ btilde, R dt, const R* __restrict__ vp,
                                                const R* __restrict__ zpi, R* __restrict__ zp, long long lb) {
  vp = lane_ptr(vp, lb);
  zpi = lane_ptr(zpi, lb);
  zp = lane_ptr(zp, lb);
  const unsigned T = blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= t.nT) return;
  const unsigned q = t.d_nx.div(T);
  const int i = (int)(T - q * (unsigned)t.nx), k = (int)t.d_ny.div(q), j = (int)(q - (unsigned)k * (unsigned)t.ny);
  R a[6], z[6];
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) {
    a[lf] = ApPi[lf * t.nT + T];
    z[lf] = zpi[t.face(i, j, k, lf)];
  }
  R c = R(0);
#pragma unroll
  for (int lf = 0; lf < 6; ++lf) c += a[lf] * z[lf];
  zp[T] = (vp[T] - dt * c) / btilde[T];
}

// t_u = v_u - A_up z_p: each node gathers its (up to) eight cells; 32-bit
// node decoding, every cell's loads issued before the sums
template <typename R>
__global__ void __launch_bounds__(256) k_prec_u(FaceTopo32 t, const R* __restrict__ Aup, const R* __restrict__ vu,
                                                const R* __restrict__ zp, R* __restrict__ tu, long long lb) {
  vu = lane_ptr(vu, lb);
  zp = lane_ptr(zp, lb);
  tu = lane_ptr(tu, lb);
  const unsigned n = blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned nN = (unsigned)(t.nx + 1) * (unsigned)(t.ny + 1) * (unsigned)(t.nz + 1);
  if (n >= nN) return;
  const unsigned r = t.d_nx1.div(n);
  const int ni = (int)(n - r * (unsigned)(t.nx + 1)), nk = (int)t.d_ny1.div(r),
            nj = (int)(r - (unsigned)nk * (unsigned)(t.ny + 1));
  R av[8][3], pv[8];
#pragma unroll
  for (int c = 0; c < 8; ++c) {  // c = dx + 2 dy + 4 dz: cell (ni - 1 + dx, nj - 1 + dy, nk - 1 + dz)
    const int cx = ni - 1 + (c & 1), cy = nj - 1 + ((c >> 1) & 1), cz = nk - 1 + (c >> 2);
    const bool in = cx >= 0 && cx < t.nx && cy >= 0 && cy < t.ny && cz >= 0 && cz < t.nz;
    const unsigned T = in ? t.cell(cx, cy, cz) : 0u;
    const int a = (ni - cx) + 2 * (nj - cy) + 4 * (nk - cz);  // local node of n in cell T
    const R p = zp[T];
    pv[c] = in ? p : R(0);
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const R v = Aup[(unsigned)(3 * a + q) * t.nT + T];
      av[c][q] = in ? v : R(0);
    }
  }
  R y0 = R(0), y1 = R(0), y2 = R(0);
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    y0 += av[c][0] * pv[c];
    y1 += av[c][1] * pv[c];
    y2 += av[c][2] * pv[c];
  }
  tu[3 * n] = vu[3 * n] - y0;
  tu[3 * n + 1] = vu[3 * n + 1] - y1;
  tu[3 * n + 2] = vu[3 * n + 2] - y2;
}

// transposed preconditioner M^T (forward substitution u, p, pi):
// z_p = B~^-1 (v_p - A_up^T z_u),  t_pi = v_pi - dt A_ppi^T z_p
template <typename R>
__global__ void k_precT_p(Dims d, const R* __restrict__ Aup, const R* __restrict__ btilde, const R* __restrict__ vp,
                          const R* __restrict__ zu, R* __restrict__ zp) {
  const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= d.nT) return;
  const int i = (int)(T % d.nx), j = (int)((T / d.nx) % d.ny), k = (int)(T / ((long long)d.nx * d.ny));
  R s = vp[T];
  for (int a = 0; a < 8; ++a) {
    const long long n = node_id(d, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
    for (int c = 0; c < 3; ++c) s -= Aup[(long long)(3 * a + c) * d.nT + T] * zu[3 * n + c];
  }
  zp[T] = s / btilde[T];
}

template <typename R>
__global__ void k_precT_pi(Dims d, const R* __restrict__ ApPi, R dt, const R* __restrict__ vpi,
                           const R* __restrict__ zp, R* __restrict__ tpi) {
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= d.nF) return;
  long long cell[2];
  int lf[2], ijk[2][3];
  face_cells(d, f, cell, lf, ijk);
  R s = R(0);
  for (int q = 0; q < 2; ++q)
    if (cell[q] >= 0) s += ApPi[(long long)lf[q] * d.nT + cell[q]] * zp[cell[q]];
  tpi[f] = vpi[f] - dt * s;
}

// g_T -= lambda^T (dA_H / d ln kappa_T) x.  With kappa_T scaled as a whole,
// W_T = A_ww,T^-1 is proportional to kappa_T, so the derivative of cell T's
// condensed flow contribution is that contribution itself:
// p row:  dt (1^T W 1 p_T - (W 1)^T pi_T);  pi rows: W pi_T - W 1 p_T
// (drained faces, whose rows and columns are eliminated, take no part).
__global__ void k_grad_logk(Dims d, const double* __restrict__ W, const double* __restrict__ W1,
                            const double* __restrict__ sW, const unsigned char* __restrict__ face_bc, double dt,
                            const double* __restrict__ lam, const double* __restrict__ x, double* __restrict__ grad) {
  const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= d.nT) return;
  const int i = (int)(T % d.nx), j = (int)((T / d.nx) % d.ny), k = (int)(T / ((long long)d.nx * d.ny));
  const long long nU = 3 * d.nN, oP = nU, oPi = nU + d.nT;
  double pi[6], lpi[6];
  for (int lf = 0; lf < 6; ++lf) {
    const long long f = cell_face(d, i, j, k, lf);
    const bool fixed = face_bc[f] & 2;
    pi[lf] = fixed ? 0.0 : x[oPi + f];
    lpi[lf] = fixed ? 0.0 : lam[oPi + f];
  }
  const double p = x[oP + T], lp = lam[oP + T];
  double w1pi = 0.0;
  for (int f = 0; f < 6; ++f) w1pi += W1[(long long)f * d.nT + T] * pi[f];
  double acc = lp * dt * (sW[T] * p - w1pi);
  for (int f = 0; f < 6; ++f) {
    double r = -W1[(long long)f * d.nT + T] * p;
    for (int g = 0; g < 6; ++g) r += W[(long long)(6 * f + g) * d.nT + T] * pi[g];
    acc += lpi[f] * r;
  }
  grad[T] -= acc;
}

// Misfit of one step: J += 1/2 sum_top (u_z - u_z*)^2 / s_u^2
//                          + 1/2 sum_cells (p - p*)^2 / s_p^2,
// g = dJ/dx (zero outside the top u_z dofs and p).  Thread per term; block
// partial sums of J, reduced in a fixed order afterwards.
__global__ void k_misfit(Dims d, const double* __restrict__ x, const double* __restrict__ uzt,
                         const double* __restrict__ pt, double wu, double wp, double* __restrict__ g,
                         double* __restrict__ part) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long ntop = (long long)(d.nx + 1) * (d.ny + 1);
  double j = 0.0;
  if (t < ntop) {
    const long long node = (long long)d.nz * ntop + t;
    const double du = x[3 * node + 2] - uzt[t];
    g[3 * node + 2] = wu * du;
    j = 0.5 * wu * du * du;
  } else if (t < ntop + d.nT) {
    const long long T = t - ntop;
    const double dp = x[3 * d.nN + T] - pt[T];
    g[3 * d.nN + T] = wp * dp;
    j = 0.5 * wp * dp * dp;
  }
  __shared__ double sh[8];
  for (int o = 16; o > 0; o >>= 1) j += __shfl_down_sync(0xffffffffu, j, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = j;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    part[blockIdx.x] = s;
  }
}

__global__ void k_sum_into(long long nb, const double* __restrict__ part, double* __restrict__ out) {
  __shared__ double sh[8];
  double v = 0.0;
  for (long long b = threadIdx.x; b < nb; b += blockDim.x) v += part[b];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += sh[w];
    out[0] += s;
  }
}

// adjoint right-hand side g + C^T lambda_next, with C x = [0; A_pu u + S_eps|T| p; 0]
// the dependence of step n's right-hand side on step n-1:
// (C^T lambda)_u = A_pu^T lambda_p = -A_up lambda_p, (C^T lambda)_p = S_eps|T| lambda_p
__global__ void k_adjoint_rhs(Dims d, const double* __restrict__ Aup, const double* __restrict__ Seps,
                              const double* __restrict__ vol, const double* __restrict__ g,
                              const double* __restrict__ lam, double* __restrict__ rhs) {
  const long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nU = 3 * d.nN;
  if (r >= nU + d.nT + d.nF) return;
  double v = g[r];
  if (lam) {
    if (r < nU) {
      const long long n = r / 3;
      const int c = (int)(r % 3);
      const int ni = (int)(n % (d.nx + 1)), nj = (int)((n / (d.nx + 1)) % (d.ny + 1)),
                nk = (int)(n / ((long long)(d.nx + 1) * (d.ny + 1)));
      for (int cz = nk - 1; cz <= nk; ++cz)
        for (int cy = nj - 1; cy <= nj; ++cy)
          for (int cx = ni - 1; cx <= ni; ++cx) {
            if (cx < 0 || cx >= d.nx || cy < 0 || cy >= d.ny || cz < 0 || cz >= d.nz) continue;
            const long long T = cell_id(d, cx, cy, cz);
            const int a = (ni - cx) + 2 * (nj - cy) + 4 * (nk - cz);
            v -= Aup[(long long)(3 * a + c) * d.nT + T] * lam[nU + T];
          }
    } else if (r < nU + d.nT) {
      const long long T = r - nU;
      v += Seps[T] * vol[T] * lam[r];
    }
  }
  rhs[r] = v;
}

// ---------------------------------------------------------------- mixed form
// Eq. (mfeSys) with continuous RT0 fluxes q, one per face oriented along the
// face's +axis: the cell's local face lf carries the sign s_lf = -1 on its
// lower side (lf even) and +1 on its upper side.  On a no-flow face q = 0:
// its row and column are zeroed and the diagonal kept.
__device__ __forceinline__ double face_sign(int lf) { return (lf & 1) ? 1.0 : -1.0; }

// per cell face: A_qp = -s_lf, A_pq = +s_lf (0 on no-flow faces); A_pp = S|T|
__global__ void k_mixed_cells(Dims d, const unsigned char* __restrict__ face_bc, const double* __restrict__ Seps,
                              const double* __restrict__ vol, double* __restrict__ Aqp, double* __restrict__ Apq,
                              double* __restrict__ Spp) {
  const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= d.nT) return;
  const int i = (int)(T % d.nx), j = (int)((T / d.nx) % d.ny), k = (int)(T / ((long long)d.nx * d.ny));
  for (int lf = 0; lf < 6; ++lf) {
    const long long f = cell_face(d, i, j, k, lf);
    const bool noflow = face_bc[f] & 4;
    Aqp[(long long)lf * d.nT + T] = noflow ? 0.0 : -face_sign(lf);
    Apq[(long long)lf * d.nT + T] = noflow ? 0.0 : face_sign(lf);
  }
  Spp[T] = Seps[T] * vol[T];
}

// A_qq in the ELL slots of the face operators (slot 0 the face itself; slot
// 1 + 5 s + q the q-th other local face of the cell on side s), from the cell
// mass matrices A_ww,T and the face signs; lumped[f] = sum of |row|.
__global__ void k_mixed_faces(Dims d, const double* __restrict__ Aww, const unsigned char* __restrict__ face_bc,
                              double* __restrict__ Aqq, double* __restrict__ lumped) {
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= d.nF) return;
  long long cell[2];
  int lf[2], ijk[2][3];
  face_cells(d, f, cell, lf, ijk);
  const bool fixed = face_bc[f] & 4;
  double diag = 0.0, lsum = 0.0;
  const long long nF = d.nF, nT = d.nT;
  for (int s = 0; s < 2; ++s) {
    if (cell[s] < 0) {
      for (int q = 0; q < 5; ++q) Aqq[(1 + 5 * s + q) * nF + f] = 0.0;
      continue;
    }
    const long long T = cell[s];
    const int l = lf[s];
    diag += Aww[(long long)(6 * l + l) * nT + T];
    int q = 0;
    for (int m = 0; m < 6; ++m) {
      if (m == l) continue;
      const long long g = cell_face(d, ijk[s][0], ijk[s][1], ijk[s][2], m);
      double v = face_sign(l) * face_sign(m) * Aww[(long long)(6 * l + m) * nT + T];
      if (fixed || (face_bc[g] & 4)) v = 0.0;
      Aqq[(1 + 5 * s + q) * nF + f] = v;
      lsum += fabs(v);
      ++q;
    }
  }
  Aqq[f] = diag;
  lumped[f] = lsum + fabs(diag);
}

// C~_p = A_pp + A_stab + diag(A_up^T diag(A_uu)^-1 A_up) - dt A_pq L^-1 A_qp
// on the cell lattice (25-point slots; the non-zeros are the cell and its six
// face neighbours): the diagonal gains dt / L_f per flowing face, a
// neighbour across face f gets -dt / L_f, a macro partner -beta_M |M|.
__global__ void k_mixed_cp(Dims d, const double* __restrict__ Auu, const double* __restrict__ Aup,
                           const double* __restrict__ Spp, const double* __restrict__ stabc,
                           const unsigned char* __restrict__ face_bc, const double* __restrict__ lumped, double dt,
                           double* __restrict__ Cp) {
  const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (T >= d.nT) return;
  const int i = (int)(T % d.nx), j = (int)((T / d.nx) % d.ny), k = (int)(T / ((long long)d.nx * d.ny));
  double fs = 0.0;
  for (int a = 0; a < 8; ++a) {
    const long long n = node_id(d, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
    for (int c = 0; c < 3; ++c) {
      const double v = Aup[(long long)(3 * a + c) * d.nT + T];
      const double dg = Auu[(long long)(13 * 9 + 4 * c) * d.nN + n];
      fs += v * v / dg;
    }
  }
  double out[25];
  for (int o = 0; o < 25; ++o) out[o] = 0.0;
  const double sx = stabc[T], sy = stabc[d.nT + T], sz = stabc[2 * d.nT + T];
  double diag = Spp[T] + (sx + sy + sz) + fs;
  // 25-point slot of the offset (dx, dy, dz) with |d|_1 <= 1: the diamond
  // order lists (0,0,-1) at 3, (0,-1,0) at 8, (-1,0,0) at 11, the cell at 12,
  // (1,0,0) at 13, (0,1,0) at 16, (0,0,1) at 21
  const int slot_of_lf[6] = {11, 13, 8, 16, 3, 21};
  for (int lf = 0; lf < 6; ++lf) {
    const long long f = cell_face(d, i, j, k, lf);
    if (face_bc[f] & 4) continue;
    const double c1 = dt / lumped[f];
    diag += c1;
    const int ax = lf >> 1, up = lf & 1;
    const int ni = i + (ax == 0 ? (up ? 1 : -1) : 0), nj = j + (ax == 1 ? (up ? 1 : -1) : 0),
              nk = k + (ax == 2 ? (up ? 1 : -1) : 0);
    if (ni < 0 || ni >= d.nx || nj < 0 || nj >= d.ny || nk < 0 || nk >= d.nz) continue;
    out[slot_of_lf[lf]] -= c1;
  }
  // macro partners (i ^ 1, j, k) ... are face neighbours
  if (sx != 0.0) out[(i & 1) ? 11 : 13] -= sx;
  if (sy != 0.0) out[(j & 1) ? 8 : 16] -= sy;
  if (sz != 0.0) out[(k & 1) ? 3 : 21] -= sz;
  out[12] = diag;
  for (int o = 0; o < 25; ++o) Cp[(long long)o * d.nT + T] = out[o];
}

Dims dims_of(const Ctx& c) {
  return Dims{c.nx, c.ny, c.nz, c.nN, c.nT, c.nF, c.nFx, c.nFy};
}

// 32-bit topology (invariant-divisor decoding of nodes, cells and faces)
FaceTopo32 topo32(const Ctx& c) { return FaceTopo32::make(c.nx, c.ny, c.nz, c.nT, c.nF, c.nFx, c.nFy); }

}  // namespace

void assemble_all(Ctx& c) {
  const Dims d = dims_of(c);
  MHFP_CUDA(cudaMemsetAsync(c.d_flag, 0, sizeof(int), c.stream));
  double* Ke = dalloc_n<double>(c, (size_t)576 * c.nT);
  c.Aup = dalloc_n<double>(c, (size_t)24 * c.nT);
  c.vol = dalloc_n<double>(c, c.nT);
  k_q1<<<grid_for(c.nT, Q1_WARPS), 32 * Q1_WARPS, 0, c.stream>>>(d, c.coords, c.E, c.nu, c.biot, Ke, c.Aup, c.vol,
                                                                 c.d_flag);
  MHFP_LAUNCH_CHECK();
  c.W = dalloc_n<double>(c, (size_t)36 * c.nT);
  c.W1 = dalloc_n<double>(c, (size_t)6 * c.nT);
  c.sW = dalloc_n<double>(c, c.nT);
  c.Abar = dalloc_n<double>(c, c.nT);
  k_rt0<<<grid_for(c.nT, 128), 128, 0, c.stream>>>(d, c.coords, c.mu, c.kappa, c.Seps, c.vol, c.dt, c.W, c.W1, c.sW,
                                                   c.Abar, c.d_flag);
  MHFP_LAUNCH_CHECK();
  c.stabc = dalloc_n<double>(c, (size_t)3 * c.nT);
  k_stab<<<grid_for(c.nT, 128), 128, 0, c.stream>>>(d, c.E, c.nu, c.biot, c.vol, c.stabc);
  MHFP_LAUNCH_CHECK();
  c.Auu.Lx = c.nx + 1; c.Auu.Ly = c.ny + 1; c.Auu.Lz = c.nz + 1;
  c.Auu.N = c.nN; c.Auu.bs = 3; c.Auu.kind = ST_BOX1;
  c.Auu.val = dalloc_n<double>(c, (size_t)27 * 9 * c.nN);
  k_assemble_uu<<<grid_for(c.nN * 27, 256), 256, 0, c.stream>>>(d, Ke, c.node_fix, c.Auu.val);
  MHFP_LAUNCH_CHECK();
  k_aup_dirichlet<<<grid_for(c.nT * 24, 256), 256, 0, c.stream>>>(d, c.node_fix, c.Aup);
  MHFP_LAUNCH_CHECK();
  c.fu = dalloc_n<double>(c, (size_t)c.nU);
  k_face_load<<<grid_for(c.nN, 128), 128, 0, c.stream>>>(d, c.coords, c.face_bc, c.node_fix, c.trac[0], c.trac[1],
                                                         c.trac[2], c.fu);
  MHFP_LAUNCH_CHECK();
  int hflag = 0;
  MHFP_CUDA(cudaMemcpyAsync(&hflag, c.d_flag, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  MHFP_CUDA(cudaStreamSynchronize(c.stream));
  // the element stiffness is consumed by the gather; release it now
  for (auto it = c.allocs.begin(); it != c.allocs.end(); ++it)
    if (*it == (void*)Ke) { c.allocs.erase(it); break; }
  MHFP_CUDA(cudaFree(Ke));
  if (hflag & 1) throw Error{MHFP_ERR_MESH, "inverted or degenerate element (det J <= 0 at a Gauss point)"};
  if (hflag & 2) throw Error{MHFP_ERR_MESH, "RT0 element mass matrix is not positive definite"};
}

// B~_p, A_ppi, the face operators A_pipi and C~_pi and the equilibration.
// Buffers are allocated on the first call; a later call (after a
// permeability update) recomputes every entry in place.
void build_preconditioner_blocks(Ctx& c) {
  const Dims d = dims_of(c);
  if (!c.btilde) c.btilde = dalloc_n<double>(c, c.nT);
  if (!c.ApPi) c.ApPi = dalloc_n<double>(c, (size_t)6 * c.nT);
  k_btilde<<<grid_for(c.nT, 128), 128, 0, c.stream>>>(d, c.Auu.val, c.Aup, c.Seps, c.vol, c.stabc, c.sW, c.W1,
                                                      c.face_bc, c.dt, c.btilde, c.ApPi);
  MHFP_LAUNCH_CHECK();
  if (!c.ell_col) {
    c.ell_col = dalloc_n<int>(c, (size_t)11 * c.nF);
    c.Apipi = dalloc_n<double>(c, (size_t)11 * c.nF);
    c.Cpi = dalloc_n<double>(c, (size_t)11 * c.nF);
    c.pw = dalloc_n<double>(c, c.nF);
  }
  k_face_ell<<<grid_for(c.nF, 128), 128, 0, c.stream>>>(d, c.W, c.W1, c.btilde, c.face_bc, c.dt, c.ell_col, c.Apipi,
                                                        c.Cpi, c.pw);
  MHFP_LAUNCH_CHECK();
  if (!c.ds) {
    c.ds = dalloc_n<double>(c, c.n);
    c.ds_inv = dalloc_n<double>(c, c.n);
  }
  k_scalings<<<grid_for(c.n, 256), 256, 0, c.stream>>>(d, c.Auu.val, c.btilde, c.Cpi, c.ds, c.ds_inv);
  MHFP_LAUNCH_CHECK();
}

namespace {
// kappa_ratio[3T + q] = kappa[3T + q] / kappa[3T] (the anisotropy the
// permeability update keeps)
__global__ void k_kappa_ratio(long long nT, const double* __restrict__ kappa, double* __restrict__ ratio) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nT) return;
  const double k0 = kappa[3 * t];
  for (int q = 0; q < 3; ++q) ratio[3 * t + q] = kappa[3 * t + q] / k0;
}

// kappa_T = exp(logk_T) * ratio_T.  Pass 0 only checks (a non-finite or
// non-positive result sets flag bit 4); pass 1, run when no cell failed,
// writes.
__global__ void k_set_kappa(long long nT, const double* __restrict__ logk, const double* __restrict__ ratio,
                            double* __restrict__ kappa, int* __restrict__ flag, int write) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nT) return;
  const double s = exp(logk[t]);
  double k[3];
  bool ok = isfinite(s) && s > 0.0;
  for (int q = 0; q < 3; ++q) {
    k[q] = s * ratio[3 * t + q];
    ok = ok && isfinite(k[q]) && k[q] > 0.0;
  }
  if (!ok) atomicOr(flag, 4);
  if (write && ok)
    for (int q = 0; q < 3; ++q) kappa[3 * t + q] = k[q];
}
}  // namespace

// New per-cell log-permeability: kappa_T = exp(logk_T) times the cell's
// create-time anisotropy ratios, then the RT0 condensation (W_T, W_T 1,
// 1^T W_T 1, Abar_pp) and the preconditioner blocks recomputed in place.
// A_uu, A_up, |T| and the stabilization do not depend on kappa.
void update_logk_blocks(Ctx& c, const double* logk) {
  const Dims d = dims_of(c);
  if (!c.kappa_ratio) {
    c.kappa_ratio = dalloc_n<double>(c, (size_t)3 * c.nT);
    k_kappa_ratio<<<grid_for(c.nT, 256), 256, 0, c.stream>>>(c.nT, c.kappa, c.kappa_ratio);
    MHFP_LAUNCH_CHECK();
  }
  MHFP_CUDA(cudaMemsetAsync(c.d_flag, 0, sizeof(int), c.stream));
  k_set_kappa<<<grid_for(c.nT, 256), 256, 0, c.stream>>>(c.nT, logk, c.kappa_ratio, c.kappa, c.d_flag, 0);
  MHFP_LAUNCH_CHECK();
  int hflag = 0;
  MHFP_CUDA(cudaMemcpyAsync(&hflag, c.d_flag, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  MHFP_CUDA(cudaStreamSynchronize(c.stream));
  if (hflag & 4) throw Error{MHFP_ERR_ARG, "log-permeability gives a non-finite or non-positive permeability"};
  k_set_kappa<<<grid_for(c.nT, 256), 256, 0, c.stream>>>(c.nT, logk, c.kappa_ratio, c.kappa, c.d_flag, 1);
  MHFP_LAUNCH_CHECK();
  k_rt0<<<grid_for(c.nT, 128), 128, 0, c.stream>>>(d, c.coords, c.mu, c.kappa, c.Seps, c.vol, c.dt, c.W, c.W1, c.sW,
                                                   c.Abar, c.d_flag);
  MHFP_LAUNCH_CHECK();
  MHFP_CUDA(cudaMemcpyAsync(&hflag, c.d_flag, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  MHFP_CUDA(cudaStreamSynchronize(c.stream));
  if (hflag & 2) throw Error{MHFP_ERR_MESH, "RT0 element mass matrix is not positive definite"};
  build_preconditioner_blocks(c);
}

// The mixed formulation's blocks (opt.formulation = 1): A_ww again from
// the RT0 element kernel, A_qq and its lumped diagonal, A_qp / A_pq per
// cell face, A_pp, C~_p on the cell lattice and the equilibration
// D_s = diag(A_uu, C~_p, A_qq)^(-1/2).
void build_mixed_blocks(Ctx& c) {
  const Dims d = dims_of(c);
  double* Aww = dalloc_n<double>(c, (size_t)36 * c.nT);
  MHFP_CUDA(cudaMemsetAsync(c.d_flag, 0, sizeof(int), c.stream));
  k_rt0<<<grid_for(c.nT, 128), 128, 0, c.stream>>>(d, c.coords, c.mu, c.kappa, c.Seps, c.vol, c.dt, c.W, c.W1, c.sW,
                                                   c.Abar, c.d_flag, Aww);
  MHFP_LAUNCH_CHECK();
  c.Aqp_c = dalloc_n<double>(c, (size_t)6 * c.nT);
  c.Apq_c = dalloc_n<double>(c, (size_t)6 * c.nT);
  c.Spp = dalloc_n<double>(c, c.nT);
  k_mixed_cells<<<grid_for(c.nT, 256), 256, 0, c.stream>>>(d, c.face_bc, c.Seps, c.vol, c.Aqp_c, c.Apq_c, c.Spp);
  MHFP_LAUNCH_CHECK();
  c.Aqq = dalloc_n<double>(c, (size_t)11 * c.nF);
  double* lumped = dalloc_n<double>(c, c.nF);
  k_mixed_faces<<<grid_for(c.nF, 128), 128, 0, c.stream>>>(d, Aww, c.face_bc, c.Aqq, lumped);
  MHFP_LAUNCH_CHECK();
  c.Cp = dalloc_n<double>(c, (size_t)25 * c.nT);
  k_mixed_cp<<<grid_for(c.nT, 128), 128, 0, c.stream>>>(d, c.Auu.val, c.Aup, c.Spp, c.stabc, c.face_bc, lumped, c.dt,
                                                        c.Cp);
  MHFP_LAUNCH_CHECK();
  if (!c.ds) {
    c.ds = dalloc_n<double>(c, c.n);
    c.ds_inv = dalloc_n<double>(c, c.n);
  }
  k_scalings<<<grid_for(c.n, 256), 256, 0, c.stream>>>(d, c.Auu.val, c.Cp + (size_t)12 * c.nT, c.Aqq, c.ds,
                                                       c.ds_inv);
  MHFP_LAUNCH_CHECK();
  int hflag = 0;
  MHFP_CUDA(cudaMemcpyAsync(&hflag, c.d_flag, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  MHFP_CUDA(cudaStreamSynchronize(c.stream));
  // the cell mass matrices are consumed by the face rows; release them now
  for (auto it = c.allocs.begin(); it != c.allocs.end(); ++it)
    if (*it == (void*)Aww) { c.allocs.erase(it); break; }
  MHFP_CUDA(cudaFree(Aww));
  if (hflag & 2) throw Error{MHFP_ERR_MESH, "RT0 element mass matrix is not positive definite"};
}

// y = A_M x (or D_s (b - A_M x)) for the mixed formulation [u | p | q]: the
// u rows as for the hybrid system; p rows A_pu x_u + (A_pp + A_stab) x_p +
// dt A_pq x_q; q rows A_qp x_p + A_qq x_q
void apply_operator_mixed(Ctx& c, const double* x, double* y, const double* so, const double* bsub) {
  const Dims d = dims_of(c);
  timing_begin(c, 1);
  k_apply_u<<<lgrid(grid_for(c.nN, APPLY_U_NODES)), dim3(APPLY_U_NODES, 3), 0, c.stream>>>(d, c.Auu.val, c.Aup, x, y, so,
                                                                                    bsub, 1.0, lbytes());
  MHFP_LAUNCH_CHECK();
  k_apply_p<<<lgrid(grid_for(c.nT, 256)), 256, 0, c.stream>>>(topo32(c), c.Aup, c.Spp, c.stabc, c.Apq_c, c.dt, x, y, so,
                                                       bsub, 1.0, lbytes());
  MHFP_LAUNCH_CHECK();
  k_apply_pi<<<lgrid(grid_for(c.nF, 256)), 256, 0, c.stream>>>(topo32(c), 3 * c.nN, c.Aqp_c, c.Aqq, x, y, so, bsub, 1.0, lbytes());
  MHFP_LAUNCH_CHECK();
  const double bytes = 27.0 * 9 * 8 * c.nN + 2.0 * 24 * 8 * c.nT + 11.0 * 8 * c.nF + 17.0 * 8 * c.nT + 16.0 * c.n;
  timing_end(c, 1, bytes);
}

// the block-triangular preconditioner's p right-hand side (Eq. prec, forward
// substitution): t_p = v_p - A_pu z_u - dt A_pq z_q
void btp_p_rhs(Ctx& c, const double* vp, const double* zu, const double* zq, double* tp) {
  k_btp_p<<<grid_for(c.nT, 256), 256, 0, c.stream>>>(topo32(c), c.Aup, c.Apq_c, c.dt, vp, zu, zq, tp);
  MHFP_LAUNCH_CHECK();
}

void build_rhs(Ctx& c, const double* xprev, double scale, double* rhs) {
  const Dims d = dims_of(c);
  k_rhs<<<grid_for(c.n, 256), 256, 0, c.stream>>>(d, c.fu, c.Aup, c.Seps, c.vol, xprev, scale, rhs);
  MHFP_LAUNCH_CHECK();
}

void apply_operator(Ctx& c, const double* x, double* y, const double* so, const double* bsub, bool transpose) {
  if (c.opt.formulation == 1) {
    if (transpose) throw Error{MHFP_ERR_STATE, "the mixed formulation has no transposed solve"};
    apply_operator_mixed(c, x, y, so, bsub);
    return;
  }
  const Dims d = dims_of(c);
  timing_begin(c, 1);
  const double sgn = transpose ? -1.0 : 1.0;
  k_apply_u<<<lgrid(grid_for(c.nN, APPLY_U_NODES)), dim3(APPLY_U_NODES, 3), 0, c.stream>>>(d, c.Auu.val, c.Aup, x, y, so,
                                                                                    bsub, sgn, lbytes());
  MHFP_LAUNCH_CHECK();
  k_apply_p<<<lgrid(grid_for(c.nT, 256)), 256, 0, c.stream>>>(topo32(c), c.Aup, c.Abar, c.stabc, c.ApPi,
                                                       transpose ? 1.0 : c.dt, x, y, so, bsub, sgn, lbytes());
  MHFP_LAUNCH_CHECK();
  k_apply_pi<<<lgrid(grid_for(c.nF, 256)), 256, 0, c.stream>>>(FaceTopo32::make(c.nx, c.ny, c.nz, c.nT, c.nF, c.nFx, c.nFy),
                                                        3 * c.nN, c.ApPi, c.Apipi, x, y, so, bsub,
                                                        transpose ? c.dt : 1.0, lbytes());
  MHFP_LAUNCH_CHECK();
  // algorithmic bytes: A_uu values (27*9 doubles/node) + A_up read twice
  // (24 doubles/cell) + ELL values (11 doubles/face; the columns are
  // computed) + p-block (~17 doubles/cell) + vectors (read x, write y: 2 * 8
  // B per dof).
  const double bytes = 27.0 * 9 * 8 * c.nN + 2.0 * 24 * 8 * c.nT + 11.0 * 8 * c.nF + 17.0 * 8 * c.nT + 16.0 * c.n;
  timing_end(c, 1, bytes);
}

void precond_p_step(Ctx& c, const double* vp, const double* zpi, double* zp) {
  const Dims d = dims_of(c);
  k_prec_p<double><<<lgrid(grid_for(c.nT, 256)), 256, 0, c.stream>>>(topo32(c), c.ApPi, c.btilde, c.dt, vp, zpi, zp, lbytes());
  MHFP_LAUNCH_CHECK();
}

void precond_u_rhs(Ctx& c, const double* vu, const double* zp, double* tu) {
  const Dims d = dims_of(c);
  k_prec_u<double><<<lgrid(grid_for(c.nN, 256)), 256, 0, c.stream>>>(topo32(c), c.Aup, vu, zp, tu, lbytes());
  MHFP_LAUNCH_CHECK();
}

void precond_p_step(Ctx& c, const float* vp, const float* zpi, float* zp) {
  const Dims d = dims_of(c);
  k_prec_p<float><<<lgrid(grid_for(c.nT, 256)), 256, 0, c.stream>>>(topo32(c), c.ApPif, c.btildef, (float)c.dt, vp, zpi,
                                                             zp, lbytes());
  MHFP_LAUNCH_CHECK();
}

void precond_u_rhs(Ctx& c, const float* vu, const float* zp, float* tu) {
  const Dims d = dims_of(c);
  k_prec_u<float><<<lgrid(grid_for(c.nN, 256)), 256, 0, c.stream>>>(topo32(c), c.Aupf, vu, zp, tu, lbytes());
  MHFP_LAUNCH_CHECK();
}

void precondT_p_step(Ctx& c, const double* vp, const double* zu, double* zp) {
  const Dims d = dims_of(c);
  k_precT_p<double><<<grid_for(c.nT, 256), 256, 0, c.stream>>>(d, c.Aup, c.btilde, vp, zu, zp);
  MHFP_LAUNCH_CHECK();
}
void precondT_p_step(Ctx& c, const float* vp, const float* zu, float* zp) {
  const Dims d = dims_of(c);
  k_precT_p<float><<<grid_for(c.nT, 256), 256, 0, c.stream>>>(d, c.Aupf, c.btildef, vp, zu, zp);
  MHFP_LAUNCH_CHECK();
}
void precondT_pi_rhs(Ctx& c, const double* vpi, const double* zp, double* tpi) {
  const Dims d = dims_of(c);
  k_precT_pi<double><<<grid_for(c.nF, 256), 256, 0, c.stream>>>(d, c.ApPi, c.dt, vpi, zp, tpi);
  MHFP_LAUNCH_CHECK();
}
void precondT_pi_rhs(Ctx& c, const float* vpi, const float* zp, float* tpi) {
  const Dims d = dims_of(c);
  k_precT_pi<float><<<grid_for(c.nF, 256), 256, 0, c.stream>>>(d, c.ApPif, (float)c.dt, vpi, zp, tpi);
  MHFP_LAUNCH_CHECK();
}
void grad_logk(Ctx& c, const double* lam, const double* x, double* grad) {
  const Dims d = dims_of(c);
  k_grad_logk<<<grid_for(c.nT, 128), 128, 0, c.stream>>>(d, c.W, c.W1, c.sW, c.face_bc, c.dt, lam, x, grad);
  MHFP_LAUNCH_CHECK();
}

void misfit(Ctx& c, const double* x, const double* uzt, const double* pt, double wu, double wp, double* J,
            double* g, double* part, long long npart) {
  const Dims d = dims_of(c);
  const long long nterm = (long long)(c.nx + 1) * (c.ny + 1) + c.nT;
  const long long nb = grid_for(nterm, 256);
  if (nb > npart) throw Error{MHFP_ERR_ARG, "misfit needs more partial sums than the workspace holds"};
  MHFP_CUDA(cudaMemsetAsync(g, 0, c.n * sizeof(double), c.stream));
  k_misfit<<<(unsigned)nb, 256, 0, c.stream>>>(d, x, uzt, pt, wu, wp, g, part);
  MHFP_LAUNCH_CHECK();
  k_sum_into<<<1, 256, 0, c.stream>>>(nb, part, J);
  MHFP_LAUNCH_CHECK();
}

void adjoint_rhs(Ctx& c, const double* g, const double* lam_next, double* rhs) {
  const Dims d = dims_of(c);
  k_adjoint_rhs<<<grid_for(c.n, 256), 256, 0, c.stream>>>(d, c.Aup, c.Seps, c.vol, g, lam_next, rhs);
  MHFP_LAUNCH_CHECK();
}

__global__ void k_cast_blocks(long long n, const double* __restrict__ x, float* __restrict__ y) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (float)x[i];
}

// FP32 copies of the blocks the mixed-precision preconditioner reads
// (allocated on the first call, overwritten in place afterwards)
void make_fp32_blocks(Ctx& c) {
  auto cast = [&](float*& dst, const double* src, long long n) {
    if (!dst) dst = dalloc_n<float>(c, n);
    k_cast_blocks<<<grid_for(n, 256), 256, 0, c.stream>>>(n, src, dst);
    MHFP_LAUNCH_CHECK();
  };
  cast(c.ApPif, c.ApPi, 6 * c.nT);
  cast(c.btildef, c.btilde, c.nT);
  cast(c.Aupf, c.Aup, 24 * c.nT);
  if (!c.tf) c.tf = dalloc_n<float>(c, c.n);
  if (!c.zf) c.zf = dalloc_n<float>(c, c.n);
  // float-float A_uu (symmetric half) and A_up for the Arnoldi step (A_uu and
  // A_up do not depend on the permeability: built once)
  if (!c.auu_h) {
    const long long N = c.nN;
    const size_t elems = (size_t)((N + 31) / 32) * 126 * 32;
    c.auu_h = dalloc_n<float>(c, elems);
    c.auu_l = dalloc_n<float>(c, elems);
    MHFP_CUDA(cudaMemsetAsync(c.auu_h, 0, elems * sizeof(float), c.stream));
    MHFP_CUDA(cudaMemsetAsync(c.auu_l, 0, elems * sizeof(float), c.stream));
    k_split_sym<<<grid_for(126 * N, 256), 256, 0, c.stream>>>(N, c.Auu.val + 13 * 9 * N, c.auu_h, c.auu_l);
    MHFP_LAUNCH_CHECK();
    c.aup_l = dalloc_n<float>(c, 24 * c.nT);
    k_split_lo<<<grid_for(24 * c.nT, 256), 256, 0, c.stream>>>(24 * c.nT, c.Aup, c.Aupf, c.aup_l);
    MHFP_LAUNCH_CHECK();
    c.pd_h = dalloc_n<float>(c, c.nT);
    c.pd_l = dalloc_n<float>(c, c.nT);
    c.st_h = dalloc_n<float>(c, 3 * c.nT);
    c.st_l = dalloc_n<float>(c, 3 * c.nT);
    c.appi_h = dalloc_n<float>(c, 6 * c.nT);
    c.appi_l = dalloc_n<float>(c, 6 * c.nT);
    c.apipi_h = dalloc_n<float>(c, 11 * c.nF);
    c.apipi_l = dalloc_n<float>(c, 11 * c.nF);
  }
  // the permeability-dependent blocks of the p and pi rows, every call
  double* pd = c.tmp_pd ? c.tmp_pd : (c.tmp_pd = dalloc_n<double>(c, c.nT));
  k_pdiag<<<grid_for(c.nT, 256), 256, 0, c.stream>>>(c.nT, c.Abar, c.stabc, pd);
  MHFP_LAUNCH_CHECK();
  auto split = [&](const double* x, float* h, float* l, long long n) {
    k_split<<<grid_for(n, 256), 256, 0, c.stream>>>(n, x, h, l);
    MHFP_LAUNCH_CHECK();
  };
  split(pd, c.pd_h, c.pd_l, c.nT);
  split(c.stabc, c.st_h, c.st_l, 3 * c.nT);
  split(c.ApPi, c.appi_h, c.appi_l, 6 * c.nT);
  split(c.Apipi, c.apipi_h, c.apipi_l, 11 * c.nF);
}

namespace {
__global__ void k_narrow_f32(long long n, const double* __restrict__ x, float* __restrict__ y) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < n) y[t] = __double2float_rn(x[t]);
}
}  // namespace
void narrow_to_f32(Ctx& c, const double* x, float* y, long long n) {
  k_narrow_f32<<<grid_for(n, 256), 256, 0, c.stream>>>(n, x, y);
  MHFP_LAUNCH_CHECK();
}

void apply_operator_arnoldi(Ctx& c, const double* z, const float* zf, double* y, const double* so, bool transpose) {
  if (!ff_krylov(c)) {
    apply_operator(c, z, y, so, nullptr, transpose);
    return;
  }
  const Dims d = dims_of(c);
  timing_begin(c, 6);
  k_apply_u_ff<<<lgrid(grid_for(c.nN, 256)), 256, 0, c.stream>>>(d, c.auu_h, c.auu_l, c.Aupf, c.aup_l, zf, y, so, nullptr,
                                                           transpose ? -1.f : 1.f, lbytes());
  MHFP_LAUNCH_CHECK();
  k_apply_p_ff<<<lgrid(grid_for(c.nT, 256)), 256, 0, c.stream>>>(topo32(c), c.Aupf, c.aup_l, c.pd_h, c.pd_l, c.st_h, c.st_l,
                                                          c.appi_h, c.appi_l, transpose ? 1.0 : c.dt, zf, y, so,
                                                          transpose ? -1.0 : 1.0, lbytes());
  MHFP_LAUNCH_CHECK();
  k_apply_pi_ff<<<lgrid(grid_for(c.nF, 256)), 256, 0, c.stream>>>(topo32(c), 3 * c.nN, c.appi_h, c.appi_l, c.apipi_h,
                                                           c.apipi_l, zf, y, so, transpose ? c.dt : 1.0, lbytes());
  MHFP_LAUNCH_CHECK();
  // algorithmic bytes, every coefficient a hi + lo pair (8 B): A_uu's
  // symmetric half (126 per node) and A_up (24 per cell) by the u rows, A_up
  // again, the p block (1 + 3) and A_ppi (6) by the p rows, A_ppi (6 per
  // cell) and A_pipi (11 per face) by the pi rows; z read in FP32, y written
  // in FP64
  const double bytes = 8.0 * (126.0 * c.nN + (24.0 + 24.0 + 4.0 + 6.0 + 6.0) * c.nT + 11.0 * c.nF) + 4.0 * c.n +
                       8.0 * c.n;
  timing_end(c, 6, bytes);
}

}  // namespace mhfp

// ============================================================================
// Residual norm without allocation.
//
// mhfp_solve checks its answer with ||D_s (b - A_H x)|| computed through the
// handle's Krylov workspace (an n-vector and a partial-sum buffer, allocated
// on the first solve).  Callers that must not trigger any device allocation
// (hosts whose device memory is handed to their own pool allocator up front,
// loops that must not allocate once running) use mhfp_residual_norm_noalloc
// instead: each row kernel below folds the operator rows straight into
// per-block partial sums that live in the file-scope array
// g_noalloc_partials, so nothing is allocated per call.
// ============================================================================
namespace mhfp {
namespace {

constexpr int NOALLOC_BLOCK = (int)NOALLOC_ROWS_PER_BLOCK;
// 2 partial sums per thread block -> NOALLOC_MAX_BLOCKS (65536) blocks = 1 MiB
// of device memory
static __device__ __align__(256) double g_noalloc_partials[2 * NOALLOC_MAX_BLOCKS];

std::mutex g_noalloc_mu;
// Per device ordinal, filled on first use.  The cached address stays valid
// for as long as the device's primary context lives; the library assumes it
// lives for the whole process (no cudaDeviceReset between calls).
double* g_noalloc_ptr[128] = {};

__device__ __forceinline__ void na_block_store(double r2, double b2, double* part, long long slot) {
  __shared__ double sr[NOALLOC_BLOCK / 32], sb[NOALLOC_BLOCK / 32];
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_down_sync(0xffffffffu, r2, o);
    b2 += __shfl_down_sync(0xffffffffu, b2, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sr[wid] = r2; sb[wid] = b2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < NOALLOC_BLOCK / 32; ++w) { a += sr[w]; c += sb[w]; }
    part[2 * slot] = a;
    part[2 * slot + 1] = c;
  }
}

// u rows of D_s (b - A_H x): A_uu x_u + A_up x_p
__global__ void __launch_bounds__(NOALLOC_BLOCK) k_na_u(Dims d, const double* __restrict__ Auu,
                                                        const double* __restrict__ Aup, const double* __restrict__ x,
                                                        const double* __restrict__ b, const double* __restrict__ ds,
                                                        double* __restrict__ part, long long slot0) {
  const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0, b2 = 0.0;
  if (n < d.nN) {
    const int ni = (int)(n % (d.nx + 1)), nj = (int)((n / (d.nx + 1)) % (d.ny + 1)),
              nk = (int)(n / ((long long)(d.nx + 1) * (d.ny + 1)));
    const long long N = d.nN;
    double y[3] = {0, 0, 0};
    for (int o = 0; o < 27; ++o) {
      const int dx = o % 3 - 1, dy = (o / 3) % 3 - 1, dz = o / 9 - 1;
      const int mi = ni + dx, mj = nj + dy, mk = nk + dz;
      if (mi < 0 || mi > d.nx || mj < 0 || mj > d.ny || mk < 0 || mk > d.nz) continue;
      const long long m = node_id(d, mi, mj, mk);
      for (int r = 0; r < 3; ++r)
        for (int s = 0; s < 3; ++s) y[r] += Auu[(long long)(o * 9 + 3 * r + s) * N + n] * x[3 * m + s];
    }
    const double* xp = x + 3 * N;
    for (int cz = nk - 1; cz <= nk; ++cz)
      for (int cy = nj - 1; cy <= nj; ++cy)
        for (int cx = ni - 1; cx <= ni; ++cx) {
          if (cx < 0 || cx >= d.nx || cy < 0 || cy >= d.ny || cz < 0 || cz >= d.nz) continue;
          const long long T = cell_id(d, cx, cy, cz);
          const int a = (ni - cx) + 2 * (nj - cy) + 4 * (nk - cz);
          for (int r = 0; r < 3; ++r) y[r] += Aup[(long long)(3 * a + r) * d.nT + T] * xp[T];
        }
    for (int r = 0; r < 3; ++r) {
      const long long row = 3 * n + r;
      const double sb = ds[row] * b[row];
      const double rr = ds[row] * (b[row] - y[r]);
      r2 += rr * rr;
      b2 += sb * sb;
    }
  }
  na_block_store(r2, b2, part, slot0 + blockIdx.x);
}

// p rows: A_pu x_u + (Abar_pp + A_stab) x_p + dt A_ppi x_pi
__global__ void __launch_bounds__(NOALLOC_BLOCK) k_na_p(Dims d, const double* __restrict__ Aup,
                                                        const double* __restrict__ Abar, const double* __restrict__ stabc,
                                                        const double* __restrict__ ApPi, double dt,
                                                        const double* __restrict__ x, const double* __restrict__ b,
                                                        const double* __restrict__ ds, double* __restrict__ part,
                                                        long long slot0) {
  const long long T = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0, b2 = 0.0;
  if (T < d.nT) {
    const int i = (int)(T % d.nx), j = (int)((T / d.nx) % d.ny), k = (int)(T / ((long long)d.nx * d.ny));
    const long long nU = 3 * d.nN;
    double s = 0.0;
    for (int a = 0; a < 8; ++a) {
      const long long n = node_id(d, i + (a & 1), j + ((a >> 1) & 1), k + ((a >> 2) & 1));
      for (int c = 0; c < 3; ++c) s -= Aup[(long long)(3 * a + c) * d.nT + T] * x[3 * n + c];
    }
    const double* xp = x + nU;
    const double cx = stabc[T], cy = stabc[d.nT + T], cz = stabc[2 * d.nT + T];
    s += (Abar[T] + (cx + cy + cz)) * xp[T];
    if (cx != 0.0) s -= cx * xp[cell_id(d, i ^ 1, j, k)];
    if (cy != 0.0) s -= cy * xp[cell_id(d, i, j ^ 1, k)];
    if (cz != 0.0) s -= cz * xp[cell_id(d, i, j, k ^ 1)];
    const double* xpi = xp + d.nT;
    double c = 0.0;
    for (int lf = 0; lf < 6; ++lf) c += ApPi[(long long)lf * d.nT + T] * xpi[cell_face(d, i, j, k, lf)];
    s += dt * c;
    const long long row = nU + T;
    const double sb = ds[row] * b[row];
    const double rr = ds[row] * (b[row] - s);
    r2 = rr * rr;
    b2 = sb * sb;
  }
  na_block_store(r2, b2, part, slot0 + blockIdx.x);
}

// pi rows: A_pip x_p + A_pipi x_pi
__global__ void __launch_bounds__(NOALLOC_BLOCK) k_na_pi(Dims d, const double* __restrict__ ApPi,
                                                         const int* __restrict__ col, const double* __restrict__ Apipi,
                                                         const double* __restrict__ x, const double* __restrict__ b,
                                                         const double* __restrict__ ds, double* __restrict__ part,
                                                         long long slot0) {
  const long long f = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  double r2 = 0.0, b2 = 0.0;
  if (f < d.nF) {
    long long cell[2];
    int lf[2], ijk[2][3];
    face_cells(d, f, cell, lf, ijk);
    const long long nU = 3 * d.nN;
    const double* xp = x + nU;
    const double* xpi = xp + d.nT;
    double s = 0.0;
    for (int q = 0; q < 2; ++q)
      if (cell[q] >= 0) s += ApPi[(long long)lf[q] * d.nT + cell[q]] * xp[cell[q]];
    for (int q = 0; q < 11; ++q) s += Apipi[(long long)q * d.nF + f] * xpi[col[(long long)q * d.nF + f]];
    const long long row = nU + d.nT + f;
    const double sb = ds[row] * b[row];
    const double rr = ds[row] * (b[row] - s);
    r2 = rr * rr;
    b2 = sb * sb;
  }
  na_block_store(r2, b2, part, slot0 + blockIdx.x);
}

// out[0] = sqrt(sum of the r^2 partials), out[1] = sqrt(sum of the (D_s b)^2 partials)
__global__ void __launch_bounds__(NOALLOC_BLOCK) k_na_final(long long nblocks, const double* __restrict__ part,
                                                            double* __restrict__ out) {
  double r2 = 0.0, b2 = 0.0;
  for (long long q = threadIdx.x; q < nblocks; q += blockDim.x) {
    r2 += part[2 * q];
    b2 += part[2 * q + 1];
  }
  __shared__ double sr[NOALLOC_BLOCK / 32], sb[NOALLOC_BLOCK / 32];
  for (int o = 16; o > 0; o >>= 1) {
    r2 += __shfl_down_sync(0xffffffffu, r2, o);
    b2 += __shfl_down_sync(0xffffffffu, b2, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sr[wid] = r2; sb[wid] = b2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0.0, c = 0.0;
    for (int w = 0; w < NOALLOC_BLOCK / 32; ++w) { a += sr[w]; c += sb[w]; }
    out[0] = sqrt(a);
    out[1] = sqrt(c);
  }
}

// Device address of g_noalloc_partials for the current device.  In host code
// the array's name is only a host-side stand-in, so the address must come
// from cudaGetSymbolAddress, once per device, with that device current.
double* noalloc_scratch(int device) {
  if (device < 0 || device >= 128) throw Error{MHFP_ERR_ARG, "device ordinal out of range"};
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_ptr[device]) {
    void* p = nullptr;
    MHFP_CUDA(cudaGetSymbolAddress(&p, g_noalloc_partials));
    g_noalloc_ptr[device] = (double*)p;
  }
  return g_noalloc_ptr[device];
}

}  // namespace

void residual_norm_noalloc(Ctx& c, const double* b, const double* x, double* out) {
  const Dims d = dims_of(c);
  const long long bu = (long long)grid_for(c.nN, NOALLOC_BLOCK);
  const long long bp = (long long)grid_for(c.nT, NOALLOC_BLOCK);
  const long long bf = (long long)grid_for(c.nF, NOALLOC_BLOCK);
  const long long need = noalloc_row_blocks(c.nx, c.ny, c.nz);
  if (need != bu + bp + bf) throw Error{MHFP_ERR_ARG, "row block count mismatch"};
  if (need > NOALLOC_MAX_BLOCKS)
    throw Error{MHFP_ERR_ARG, "problem too large for the static scratch of mhfp_residual_norm_noalloc (" +
                                  std::to_string(need) + " row blocks > 65536)"};
  double* part = noalloc_scratch(c.device);
  k_na_u<<<(unsigned)bu, NOALLOC_BLOCK, 0, c.stream>>>(d, c.Auu.val, c.Aup, x, b, c.ds, part, 0);
  MHFP_LAUNCH_CHECK();
  k_na_p<<<(unsigned)bp, NOALLOC_BLOCK, 0, c.stream>>>(d, c.Aup, c.Abar, c.stabc, c.ApPi, c.dt, x, b, c.ds, part, bu);
  MHFP_LAUNCH_CHECK();
  k_na_pi<<<(unsigned)bf, NOALLOC_BLOCK, 0, c.stream>>>(d, c.ApPi, c.ell_col, c.Apipi, x, b, c.ds, part, bu + bp);
  MHFP_LAUNCH_CHECK();
  k_na_final<<<1, NOALLOC_BLOCK, 0, c.stream>>>(bu + bp + bf, part, out);
  MHFP_LAUNCH_CHECK();
}

}  // namespace mhfp
