// The paper's representation and kernel, for comparison on the same GPU (Sec. 2): D stored in
// coordinate format (Row, Col, Val arrays of its non-zeros) and the sparse matrix-vector product
// out[Row[k]] += Val[k] * in[Col[k]], one thread per non-zero k with atomic accumulation (the
// ND-range form of the paper's loop). Rows and columns index the canonical vector
// (12 * site + 3 * spin + colour); each row holds 49 non-zeros: the unit diagonal, then for each
// direction mu the forward and the backward hop, each with the two non-zero spin entries of its
// projector times the 3 colour entries of its link.
#include <cstring>

#include "../../include/wd.h"
#include "wd_device.cuh"
#include "wd_internal.h"

namespace wdk {

// Spin projectors (1 + S gamma_mu), chiral basis, as 4x4 complex tables built on the host from
// gamma_mu = [[0, B_mu], [B_mu^dag, 0]].
struct ProjTables {
  double re[2][4][4][4];  // [S = -1 (index 0) or +1 (index 1)][mu][alpha][beta]
  double im[2][4][4][4];
};

static void build_projectors(ProjTables& t) {
  // B_mu (2x2, one non-zero per row): (column, re, im) per row
  const int bcol[4][2] = {{1, 0}, {1, 0}, {0, 1}, {0, 1}};
  const double bre[4][2] = {{0, 0}, {-1, 1}, {0, 0}, {1, 1}};
  const double bim[4][2] = {{-1, -1}, {0, 0}, {-1, 1}, {0, 0}};
  memset(&t, 0, sizeof(t));
  for (int mu = 0; mu < 4; ++mu) {
    double gre[4][4] = {{0}}, gim[4][4] = {{0}};
    for (int a = 0; a < 2; ++a) {
      const int b = bcol[mu][a];
      gre[a][2 + b] = bre[mu][a];  // upper-right block B
      gim[a][2 + b] = bim[mu][a];
      gre[2 + b][a] = bre[mu][a];  // lower-left block B^dag: (B^dag)[b][a] = conj(B[a][b])
      gim[2 + b][a] = -bim[mu][a];
    }
    for (int si = 0; si < 2; ++si) {
      const double S = si ? 1.0 : -1.0;
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          t.re[si][mu][a][b] = (a == b ? 1.0 : 0.0) + S * gre[a][b];
          t.im[si][mu][a][b] = S * gim[a][b];
        }
    }
  }
}

__constant__ ProjTables c_proj;

// One thread per row (site n, spin alpha, colour A): writes its 49 entries at 49 * row.
__global__ void coo_build_kernel(Geom g, const double2* __restrict__ U /* canonical [V][4][9] */, double kappa,
                                 int* __restrict__ row, int* __restrict__ col, double2* __restrict__ val) {
  const int rw = blockIdx.x * blockDim.x + threadIdx.x;
  if (rw >= 12 * g.V) return;
  const int n = rw / 12, alpha = (rw % 12) / 3, A = rw % 3;
  int c[4];
  int r = n;
  c[0] = r % g.L[0];
  r /= g.L[0];
  c[1] = r % g.L[1];
  r /= g.L[1];
  c[2] = r % g.L[2];
  c[3] = r / g.L[2];
  size_t k = (size_t)rw * 49;
  row[k] = rw;
  col[k] = rw;
  val[k] = make_double2(1.0, 0.0);
  ++k;
  for (int mu = 0; mu < 4; ++mu) {
    for (int dir = 0; dir < 2; ++dir) {  // 0: forward (1 - gamma), U_mu(n); 1: backward (1 + gamma), U_mu(n-mu)^dag
      int nb[4] = {c[0], c[1], c[2], c[3]};
      bool wrap;
      if (dir == 0) {
        wrap = nb[mu] == g.L[mu] - 1;
        nb[mu] = wrap ? 0 : nb[mu] + 1;
      } else {
        wrap = nb[mu] == 0;
        nb[mu] = wrap ? g.L[mu] - 1 : nb[mu] - 1;
      }
      const int m = nb[0] + g.L[0] * (nb[1] + g.L[1] * (nb[2] + g.L[2] * nb[3]));
      const double phase = (wrap && g.bc[mu] < 0) ? -1.0 : 1.0;
      const int si = dir == 0 ? 0 : 1;
      const int ln = dir == 0 ? n : m;  // site whose link is used
      for (int beta = 0; beta < 4; ++beta) {
        const double pr = c_proj.re[si][mu][alpha][beta], pi = c_proj.im[si][mu][alpha][beta];
        if (pr == 0.0 && pi == 0.0) continue;
        for (int B = 0; B < 3; ++B) {
          // link entry: U[A][B] forward, (U^dag)[A][B] = conj(U[B][A]) backward
          double2 u = dir == 0 ? U[((size_t)ln * 4 + mu) * 9 + 3 * A + B] : U[((size_t)ln * 4 + mu) * 9 + 3 * B + A];
          if (dir == 1) u.y = -u.y;
          const double fr = -kappa * phase;
          // val = fr * P[alpha][beta] * u
          row[k] = rw;
          col[k] = 12 * m + 3 * beta + B;
          val[k] = make_double2(fr * (pr * u.x - pi * u.y), fr * (pr * u.y + pi * u.x));
          ++k;
        }
      }
    }
  }
}

// The paper's SpMV: one thread per non-zero, atomic accumulation into out (zeroed first).
__global__ void coo_spmv_kernel(long long nnz, const int* __restrict__ row, const int* __restrict__ col,
                                const double2* __restrict__ val, const double2* __restrict__ in, double* out) {
  const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const double2 v = val[k], x = in[col[k]];
  double* o = out + 2 * (size_t)row[k];
  atomicAdd(o, v.x * x.x - v.y * x.y);
  atomicAdd(o + 1, v.x * x.y + v.y * x.x);
}

cudaError_t launch_coo_build(const GeomH& gh, const double* U, double kappa, int* row, int* col, double* val,
                             cudaStream_t st) {
  static ProjTables tables;
  static bool built = false;
  if (!built) {
    build_projectors(tables);
    built = true;
  }
  cudaError_t e = cudaMemcpyToSymbolAsync(c_proj, &tables, sizeof(tables), 0, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  Geom g;
  memcpy(&g, &gh, sizeof(g));
  const int rows = 12 * gh.V;
  coo_build_kernel<<<(rows + 127) / 128, 128, 0, st>>>(g, reinterpret_cast<const double2*>(U), kappa, row, col,
                                                       reinterpret_cast<double2*>(val));
  return cudaGetLastError();
}

cudaError_t launch_coo_spmv(long long nnz, const int* row, const int* col, const double* val, const double* in,
                            double* out, long long nrows, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * 2 * (size_t)nrows, st);
  if (e != cudaSuccess) return e;
  const int block = 256;
  coo_spmv_kernel<<<(unsigned)((nnz + block - 1) / block), block, 0, st>>>(
      nnz, row, col, reinterpret_cast<const double2*>(val), reinterpret_cast<const double2*>(in), out);
  return cudaGetLastError();
}

}  // namespace wdk
