// Gradient gathers of the differentiable solve.  For x = A^{-1} b and the
// adjoint state lam = A^{-1} dL/dx (A symmetric):
//   stencil face f between cells i and j:  dL/dk_f = -(lam_i - lam_j)(x_i - x_j)
//     (a boundary face of cell i has j outside the grid, where lam = x = 0);
//   CSR entry (i, j):                      dL/dA_ij = -lam_i x_j.
// One thread per face (or stored entry); coalesced along x.
#include "sscg_internal.cuh"

namespace sscg {

namespace {

constexpr int kAdjThreads = 256;

// Face (c0, c1, m) along `axis` of a grid whose cells are (z, y, x), x fastest:
// it separates cells m-1 and m along that axis.
template <int AXIS>
__global__ void __launch_bounds__(kAdjThreads) face_grad_kernel(Operator A, const double* __restrict__ lam,
                                                                const double* __restrict__ x,
                                                                double* __restrict__ g) {
  const int nx = A.nx, ny = A.ny, nz = A.nz;
  const int fx = AXIS == 0 ? nx + 1 : nx;
  const int fy = AXIS == 1 ? ny + 1 : ny;
  const int fz = AXIS == 2 ? nz + 1 : nz;
  const int64_t total = (int64_t)fx * fy * fz;
  const int64_t stride = AXIS == 0 ? 1 : (AXIS == 1 ? (int64_t)nx : (int64_t)nx * ny);
  for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total; f += (int64_t)gridDim.x * blockDim.x) {
    const int ix = (int)(f % fx);
    const int64_t t = f / fx;
    const int iy = (int)(t % fy);
    const int iz = (int)(t / fy);
    const int m = AXIS == 0 ? ix : (AXIS == 1 ? iy : iz);
    const int nax = AXIS == 0 ? nx : (AXIS == 1 ? ny : nz);
    // cell with coordinate m along the axis (the "high" side) and its low neighbour
    const int cx = AXIS == 0 ? 0 : ix, cy = AXIS == 1 ? 0 : iy, cz = AXIS == 2 ? 0 : iz;
    const int64_t base = ((int64_t)cz * ny + cy) * nx + cx;  // cell with axis coordinate 0
    double lh = 0.0, xh = 0.0, ll = 0.0, xl = 0.0;
    if (m < nax) {
      const int64_t c = base + (int64_t)m * stride;
      lh = lam[c];
      xh = x[c];
    }
    if (m > 0) {
      const int64_t c = base + (int64_t)(m - 1) * stride;
      ll = lam[c];
      xl = x[c];
    }
    g[f] = -((lh - ll) * (xh - xl));
  }
}

__global__ void __launch_bounds__(kAdjThreads) csr_grad_kernel(Operator A, const double* __restrict__ lam,
                                                               const double* __restrict__ x,
                                                               double* __restrict__ g) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < A.n; i += (int64_t)gridDim.x * blockDim.x) {
    const double li = lam[i];
    for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) g[k] = -(li * x[A.col[k]]);
  }
}

int adj_grid(int64_t n) {
  int64_t g = (n + kAdjThreads - 1) / kAdjThreads;
  if (g > 152 * 16) g = 152 * 16;
  return g < 1 ? 1 : (int)g;
}

}  // namespace

cudaError_t launch_face_grad(const Operator& A, const double* lam, const double* x, double* gkx, double* gky,
                             double* gkz, cudaStream_t st) {
  const int64_t nx = A.nx, ny = A.ny, nz = A.nz;
  face_grad_kernel<0><<<adj_grid((nx + 1) * ny * nz), kAdjThreads, 0, st>>>(A, lam, x, gkx);
  face_grad_kernel<1><<<adj_grid(nx * (ny + 1) * nz), kAdjThreads, 0, st>>>(A, lam, x, gky);
  if (A.dim == 3) face_grad_kernel<2><<<adj_grid(nx * ny * (nz + 1)), kAdjThreads, 0, st>>>(A, lam, x, gkz);
  return cudaGetLastError();
}

cudaError_t launch_csr_grad(const Operator& A, const double* lam, const double* x, double* gval, cudaStream_t st) {
  csr_grad_kernel<<<adj_grid(A.n), kAdjThreads, 0, st>>>(A, lam, x, gval);
  return cudaGetLastError();
}

}  // namespace sscg
