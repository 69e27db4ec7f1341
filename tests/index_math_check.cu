// Host-side check of the library's 32-bit index arithmetic (no GPU needed):
// multiply-high division by invariant integers (Div32) against plain
// division, and the face topology (FaceTopo32) against definitions written
// out here with 64-bit arithmetic: the face numbering by family, the two
// cells of a face, and the 11 columns of a face-operator row in the slot
// order of the stored ELL (slot 0 the face itself; slot 1 + 5 s + q the q-th
// local face other than f of the cell on side s, in local-face order; f
// itself where that cell is absent).  Prints "ok" and returns 0, or prints
// the first mismatch and returns 1.
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "../paper_2002_09603_gb300/csrc/common.cuh"

using mhfp::Div32;
using mhfp::FaceTopo32;

namespace {

int fail(const char* what, long long a, long long b, long long c) {
  std::printf("mismatch: %s (%lld, %lld, %lld)\n", what, a, b, c);
  return 1;
}

// face number of local face lf of cell (i, j, k): x-faces first, then y, then
// z; local face 2a is on the - side of axis a, 2a+1 on the + side
long long ref_face(int nx, int ny, int nz, int i, int j, int k, int lf) {
  const long long nFx = (long long)(nx + 1) * ny * nz, nFy = (long long)nx * (ny + 1) * nz;
  const int a = lf / 2, up = lf % 2;
  if (a == 0) return (i + up) + (long long)(nx + 1) * (j + (long long)ny * k);
  if (a == 1) return nFx + i + (long long)nx * ((j + up) + (long long)(ny + 1) * k);
  return nFx + nFy + i + (long long)nx * (j + (long long)ny * (k + up));
}

int check_div() {
  std::vector<unsigned> ds;
  for (unsigned d = 1; d <= 300; ++d) ds.push_back(d);
  for (unsigned d : {1000u, 4225u, 65537u, 1u << 20, 2147483647u, 4294967295u}) ds.push_back(d);
  unsigned long long state = 88172645463325252ull;
  for (unsigned d : ds) {
    const Div32 q = Div32::make(d);
    for (unsigned n = 0; n < 5000; ++n)
      if (q.div(n) != n / d) return fail("Div32", d, n, q.div(n));
    for (int r = 0; r < 20000; ++r) {
      state ^= state << 13; state ^= state >> 7; state ^= state << 17;
      const unsigned n = (unsigned)state;
      if (q.div(n) != n / d) return fail("Div32", d, n, q.div(n));
    }
    for (unsigned n : {4294967295u, 4294967294u, 2147483648u, 2147483647u})
      if (q.div(n) != n / d) return fail("Div32", d, n, q.div(n));
  }
  return 0;
}

int check_faces(int nx, int ny, int nz) {
  const long long nT = (long long)nx * ny * nz;
  const long long nFx = (long long)(nx + 1) * ny * nz, nFy = (long long)nx * (ny + 1) * nz;
  const long long nF = nFx + nFy + (long long)nx * ny * (nz + 1);
  const FaceTopo32 t = FaceTopo32::make(nx, ny, nz, nT, nF, nFx, nFy);
  // cells of every face from the cells' side: owner[f][s] = cell on side s
  // (s = 0: f is the cell's + face; s = 1: its - face) and its local face
  std::vector<long long> own_cell(2 * nF, -1);
  std::vector<int> own_lf(2 * nF, -1), own_ijk(6 * nF, 0);
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j)
      for (int i = 0; i < nx; ++i) {
        const long long T = i + (long long)nx * (j + (long long)ny * k);
        if ((long long)t.cell(i, j, k) != T) return fail("cell", i, j, k);
        for (int lf = 0; lf < 6; ++lf) {
          const long long f = ref_face(nx, ny, nz, i, j, k, lf);
          if ((long long)t.face(i, j, k, lf) != f) return fail("face", T, lf, f);
          const int s = (lf % 2 == 1) ? 0 : 1;
          if (own_cell[2 * f + s] != -1) return fail("face owned twice", f, s, T);
          own_cell[2 * f + s] = T;
          own_lf[2 * f + s] = lf;
          own_ijk[6 * f + 3 * s] = i; own_ijk[6 * f + 3 * s + 1] = j; own_ijk[6 * f + 3 * s + 2] = k;
        }
      }
  for (long long f = 0; f < nF; ++f) {
    int c[2][3], lf[2];
    bool ok[2];
    t.cells((unsigned)f, c, ok, lf);
    unsigned col[11];
    t.ell_cols((unsigned)f, col);
    if (col[0] != (unsigned)f) return fail("ell slot 0", f, col[0], 0);
    for (int s = 0; s < 2; ++s) {
      const bool has = own_cell[2 * f + s] >= 0;
      if (ok[s] != has) return fail("cell presence", f, s, has);
      if (has) {
        if (lf[s] != own_lf[2 * f + s]) return fail("local face", f, s, lf[s]);
        for (int a = 0; a < 3; ++a)
          if (c[s][a] != own_ijk[6 * f + 3 * s + a]) return fail("cell index", f, s, a);
      }
      int q = 0;
      for (int m = 0; m < 6; ++m) {
        if (has && m == own_lf[2 * f + s]) continue;
        if (q == 5) break;
        const long long expect = has ? ref_face(nx, ny, nz, own_ijk[6 * f + 3 * s], own_ijk[6 * f + 3 * s + 1],
                                                own_ijk[6 * f + 3 * s + 2], m)
                                     : f;
        if ((long long)col[1 + 5 * s + q] != expect) return fail("ell column", f, 1 + 5 * s + q, expect);
        ++q;
      }
    }
  }
  return 0;
}

// Row blocks of the no-allocation residual norm against a count written out
// here (ceil of rows / 256 for nodes, cells and faces), and the acceptance
// rule at its edge: 149^3 fits in the 65536 static slots, 150^3 does not, and
// a mesh needing exactly 65536 blocks is accepted while 65537 is not.
int check_noalloc_blocks() {
  auto ceil256 = [](long long v) { return (v + 255) / 256; };
  auto ref = [&](long long nx, long long ny, long long nz) {
    const long long nodes = (nx + 1) * (ny + 1) * (nz + 1), cells = nx * ny * nz;
    const long long faces = (nx + 1) * ny * nz + nx * (ny + 1) * nz + nx * ny * (nz + 1);
    return ceil256(nodes) + ceil256(cells) + ceil256(faces);
  };
  const long long cases[][3] = {{1, 1, 1}, {6, 5, 4}, {64, 64, 64}, {128, 128, 128}, {149, 149, 149},
                                {150, 150, 150}, {1000, 3, 2}, {255, 1, 1}, {256, 1, 1}};
  for (const auto& c : cases)
    if (mhfp::noalloc_row_blocks(c[0], c[1], c[2]) != ref(c[0], c[1], c[2]))
      return fail("noalloc row blocks", c[0], c[1], c[2]);
  if (mhfp::noalloc_row_blocks(128, 128, 128) != 41346) return fail("noalloc 128^3", 41346, 0, 0);
  if (mhfp::noalloc_row_blocks(149, 149, 149) > mhfp::NOALLOC_MAX_BLOCKS) return fail("noalloc 149^3 rejected", 0, 0, 0);
  if (mhfp::noalloc_row_blocks(150, 150, 150) <= mhfp::NOALLOC_MAX_BLOCKS) return fail("noalloc 150^3 accepted", 0, 0, 0);
  // find meshes (nx, 1, 1) whose count lands exactly on the limit and one past it
  bool at = false, past = false;
  for (long long nx = 1; nx < 10000000 && !(at && past); ++nx) {
    const long long b = mhfp::noalloc_row_blocks(nx, 1, 1);
    if (b == mhfp::NOALLOC_MAX_BLOCKS) at = true;
    if (b == mhfp::NOALLOC_MAX_BLOCKS + 1) past = true;
  }
  if (!at || !past) return fail("noalloc edge cases not reached", at, past, 0);
  if (mhfp::NOALLOC_MAX_BLOCKS != 65536) return fail("noalloc slots", mhfp::NOALLOC_MAX_BLOCKS, 0, 0);
  return 0;
}

}  // namespace

int main() {
  if (check_div()) return 1;
  if (check_noalloc_blocks()) return 1;
  const int dims[][3] = {{1, 1, 1}, {2, 3, 4}, {5, 4, 3}, {7, 1, 2}, {1, 6, 1}, {10, 4, 7}, {16, 16, 16}, {9, 13, 5}};
  for (const auto& d : dims)
    if (check_faces(d[0], d[1], d[2])) return 1;
  std::printf("ok\n");
  return 0;
}
