// Approximate geodesic distances by the heat method (Crane et al. 2013), the distance source of the
// paper's experiments (Sec. 4), for many sources at once in the block layout of the CG solver
// (a column per source, chunks of up to 512).
//
//  1. Heat step (D + t L) u = delta_s, t = m h^2.  u decays geometrically with the edge distance
//     from s, so the normalised gradient of step 2 needs u to small *relative* error everywhere,
//     also where it is 1e-100.  CG only gives absolute accuracy (the far field would be noise), so
//     the step is Jacobi's iteration u <- u + w ((delta + t A u) / (D + t V) - u).  With positive
//     cotangent weights D + t L is diagonally dominant with non-positive off-diagonal entries,
//     w = 1 and every term of the series is non-negative: no cancellation.  Obtuse triangles give
//     negative weights; when the Gershgorin radius gamma = max_i t sum_j |A_ij| / (D_i + t V_i)
//     reaches 1, w = 2 / (2 + gamma) keeps the iteration convergent (D + t L is SPD and the
//     eigenvalues of its Jacobi-scaled form lie in (0, 1 + gamma]).  The sweeps stop when the
//     largest relative change of any entry is below 1e-15; a vertex the heat front is just reaching
//     changes by a large fraction, so they cannot stop before every vertex has been reached.  A
//     non-finite iterate stops them with an error.
//  2. X = -grad u / |grad u| on every triangle, and
//  3. its integrated divergence at the vertices: a warp per (triangle, 32-column slab), a lane per
//     source, FP64 atomics.
//  4. L phi = -div X by block-CG (Jacobi, FP64 refinement), with vertex 0 pinned (phi_0 = 0): the
//     divergence sums to zero, so the pinned system solves the whole one; then
//     d_s = phi - phi(s).
// FP64 throughout (the heat step in FP64 for its range; the Poisson solve as the options say).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "internal.cuh"

namespace sbha {

namespace {

constexpr int BW = 32;
constexpr int kHeatChunk = 512;
constexpr int kSweepsPerCheck = 8;
constexpr int kMaxSweeps = 200000;
constexpr double kSweepTol = 1e-15;

__global__ void k_sum(int64_t n, const double* __restrict__ x, double* __restrict__ out) {
  double s = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) s += x[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

__global__ void k_check_sources(int64_t n, int32_t ns, const int32_t* __restrict__ src, int* __restrict__ err) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < ns; i += (int64_t)gridDim.x * blockDim.x)
    if (src[i] < 0 || src[i] >= n) atomicExch(err, DERR_BAD_INDEX);
}

// Poisson matrix: L = V - A with vertex 0 pinned (row 0 the identity, column 0 dropped elsewhere),
// the diagonal stored, columns ascending.
__global__ void k_lp_count(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           int32_t* __restrict__ cnt) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int a = rowptr[i], e = rowptr[i + 1];
    cnt[i] = i == 0 ? 1 : (e - a) + 1 - ((e > a && col[a] == 0) ? 1 : 0);
  }
}

__global__ void k_lp_fill(int64_t n, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          const double* __restrict__ A, const double* __restrict__ V,
                          const int32_t* __restrict__ lrowptr, int32_t* __restrict__ lcol, double* __restrict__ lval) {
  for (int64_t ii = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; ii < n; ii += (int64_t)gridDim.x * blockDim.x) {
    const int i = static_cast<int>(ii);
    int q = lrowptr[i];
    if (i == 0) {
      lcol[q] = 0;
      lval[q] = 1.0;
      continue;
    }
    bool diag = false;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) {
      const int j = col[e];
      if (j == 0) continue;
      if (!diag && j > i) {
        lcol[q] = i;
        lval[q++] = V[i];
        diag = true;
      }
      lcol[q] = j;
      lval[q++] = -A[e];
    }
    if (!diag) {
      lcol[q] = i;
      lval[q] = V[i];
    }
  }
}

// Gershgorin radius of the Jacobi-scaled heat matrix: max_i t sum_j |A_ij| / (D_i + t V_i) into *out.
__global__ void k_heat_gamma(int64_t n, const int32_t* __restrict__ rowptr, const double* __restrict__ A,
                             const double* __restrict__ D, const double* __restrict__ V, double t,
                             unsigned long long* __restrict__ out) {
  double worst = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = rowptr[i]; e < rowptr[i + 1]; ++e) s += fabs(A[e]);
    worst = fmax(worst, t * s / (D[i] + t * V[i]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, static_cast<unsigned long long>(__double_as_longlong(worst)));
}

// One damped Jacobi sweep of (D + t L) u = delta (y = A u of the previous iterate); the largest
// relative change goes to *chg (non-negative doubles order like their bit patterns; a non-finite
// iterate records infinity).
__global__ void k_heat_sweep(int64_t n, int nb, int ncols, const int32_t* __restrict__ src, double t, double w,
                             const double* __restrict__ D, const double* __restrict__ V, const double* __restrict__ y,
                             double* __restrict__ u, unsigned long long* __restrict__ chg) {
  const int64_t total = static_cast<int64_t>(nb) * n * BW;
  double worst = 0.0;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int lane = static_cast<int>(k % BW);
    const int64_t row = k / BW;
    const int64_t v = row % n;
    const int q = static_cast<int>(row / n) * BW + lane;
    if (q >= ncols) continue;
    const double uo = u[k];
    const double un = uo + w * (((v == src[q] ? 1.0 : 0.0) + t * y[k]) / (D[v] + t * V[v]) - uo);
    const double rel = un != 0.0 ? fabs(un - uo) / fabs(un) : (uo != 0.0 ? 1.0 : 0.0);
    worst = isfinite(un) ? fmax(worst, rel) : INFINITY;
    u[k] = un;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
  if ((threadIdx.x & 31) == 0 && worst > 0.0) atomicMax(chg, static_cast<unsigned long long>(__double_as_longlong(worst)));
}

__device__ __forceinline__ double3 sub3(double3 a, double3 b) { return make_double3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ double dot3(double3 a, double3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ double3 cross3(double3 a, double3 b) {
  return make_double3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ double cot_at(double3 p, double3 q, double3 r) {  // angle at r between r->p, r->q
  double3 a = sub3(p, r), b = sub3(q, r);
  double3 cr = cross3(a, b);
  return dot3(a, b) / sqrt(dot3(cr, cr));
}

// div X at the vertices, X = -grad u / |grad u| per triangle: a warp per (triangle, slab).
__global__ void k_heat_div(int64_t nf, int64_t n, int nb, const int32_t* __restrict__ faces,
                           const double* __restrict__ xyz, const double* __restrict__ u, double* __restrict__ div) {
  const int lane = threadIdx.x & 31;
  const int64_t items = nf * nb;
  for (int64_t w = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; w < items;
       w += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t f = w % nf, slab = w / nf;
    const int a = faces[3 * f], b = faces[3 * f + 1], c = faces[3 * f + 2];
    const double3 xa = make_double3(xyz[3 * a], xyz[3 * a + 1], xyz[3 * a + 2]);
    const double3 xb = make_double3(xyz[3 * b], xyz[3 * b + 1], xyz[3 * b + 2]);
    const double3 xc = make_double3(xyz[3 * c], xyz[3 * c + 1], xyz[3 * c + 2]);
    const double3 nrm = cross3(sub3(xb, xa), sub3(xc, xa));
    const double tw = sqrt(dot3(nrm, nrm));  // twice the area
    if (!(tw > 0.0)) continue;
    const double3 N = make_double3(nrm.x / tw, nrm.y / tw, nrm.z / tw);
    const int64_t base = slab * n * BW + lane;
    const double ua = u[base + static_cast<int64_t>(a) * BW], ub = u[base + static_cast<int64_t>(b) * BW],
                 uc = u[base + static_cast<int64_t>(c) * BW];
    // grad u = 1/(2 area) sum_i u_i N x e_i, e_i the edge opposite vertex i, counter-clockwise
    const double3 ga = cross3(N, sub3(xc, xb)), gb = cross3(N, sub3(xa, xc)), gc = cross3(N, sub3(xb, xa));
    double3 g = make_double3((ua * ga.x + ub * gb.x + uc * gc.x) / tw, (ua * ga.y + ub * gb.y + uc * gc.y) / tw,
                             (ua * ga.z + ub * gb.z + uc * gc.z) / tw);
    const double gn = sqrt(dot3(g, g));
    const double3 X = gn > 0.0 ? make_double3(-g.x / gn, -g.y / gn, -g.z / gn) : make_double3(0.0, 0.0, 0.0);
    const double ca = cot_at(xb, xc, xa), cb = cot_at(xc, xa, xb), cc = cot_at(xa, xb, xc);
    atomicAdd(div + base + static_cast<int64_t>(a) * BW,
              0.5 * (cc * dot3(sub3(xb, xa), X) + cb * dot3(sub3(xc, xa), X)));
    atomicAdd(div + base + static_cast<int64_t>(b) * BW,
              0.5 * (ca * dot3(sub3(xc, xb), X) + cc * dot3(sub3(xa, xb), X)));
    atomicAdd(div + base + static_cast<int64_t>(c) * BW,
              0.5 * (cb * dot3(sub3(xa, xc), X) + ca * dot3(sub3(xb, xc), X)));
  }
}

// Poisson right-hand side -div X, the pinned row of vertex 0 cleared (in place).
__global__ void k_heat_rhs(int64_t n, int nb, double* __restrict__ b) {
  const int64_t total = static_cast<int64_t>(nb) * n * BW;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x)
    b[k] = ((k / BW) % n == 0) ? 0.0 : -b[k];
}

// D[q][v] = phi[v][q] - phi[src_q][q] (D row-major over the chunk's sources).
__global__ void k_heat_out(int64_t n, int ncols, const int32_t* __restrict__ src, const double* __restrict__ phi,
                           double* __restrict__ D) {
  const int64_t total = static_cast<int64_t>(ncols) * n;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int q = static_cast<int>(k / n);
    const int64_t v = k % n;
    const int64_t slab = (q / BW) * n;
    const int lane = q % BW;
    D[k] = phi[(slab + v) * BW + lane] - phi[(slab + src[q]) * BW + lane];
  }
}

}  // namespace

SpdReport heat_geodesics(Ctx& c, const DevMesh& m, const DevGraph& g, const int32_t* src, int32_t ns, double mfac,
                         const sbha_opts& o, double* D, int32_t* jacobi_iterations) {
  SpdReport rep;
  const int64_t n = g.n;
  const int T = 256;
  k_check_sources<<<grid_for(ns, T), T, 0, c.stream>>>(n, ns, src, c.d_err);
  c.launched("check_sources");
  c.check_device("heat_geodesics");
  // t = m h^2, h the mean edge length (every edge is listed twice)
  double* acc = c.zeros<double>(1);
  k_sum<<<grid_for(g.nnz, T), T, 0, c.stream>>>(g.nnz, g.len, acc);
  c.launched("edge_sum");
  double hsum = 0.0;
  SBHA_CUDA(cudaMemcpyAsync(&hsum, acc, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  const double h = hsum / static_cast<double>(std::max<int64_t>(g.nnz, 1));
  const double t = mfac * h * h;
  unsigned long long* chg = c.alloc<unsigned long long>(1);
  SBHA_CUDA(cudaMemsetAsync(chg, 0, sizeof(unsigned long long), c.stream));
  k_heat_gamma<<<grid_for(n, T), T, 0, c.stream>>>(n, g.rowptr, g.A, g.D, g.V, t, chg);
  c.launched("heat_gamma");
  unsigned long long gbits = 0;
  SBHA_CUDA(cudaMemcpyAsync(&gbits, chg, sizeof(gbits), cudaMemcpyDeviceToHost, c.stream));
  c.sync();
  double gamma = 0.0;
  std::memcpy(&gamma, &gbits, sizeof(gamma));
  const double w = gamma < 1.0 ? 1.0 : 2.0 / (2.0 + gamma);
  // the pinned Poisson matrix
  int32_t* cnt = c.alloc<int32_t>(n);
  k_lp_count<<<grid_for(n, T), T, 0, c.stream>>>(n, g.rowptr, g.col, cnt);
  c.launched("lp_count");
  int32_t* lrowptr = c.alloc<int32_t>(n + 1);
  const int64_t lnnz = exclusive_scan(c, cnt, lrowptr, n);
  int32_t* lcol = c.alloc<int32_t>(lnnz);
  double* lval = c.alloc<double>(lnnz);
  k_lp_fill<<<grid_for(n, T), T, 0, c.stream>>>(n, g.rowptr, g.col, g.A, g.V, lrowptr, lcol, lval);
  c.launched("lp_fill");
  c.free(cnt);
  const int C = std::min(kHeatChunk, (ns + BW - 1) / BW * BW);
  const int nb = C / BW;
  const size_t blk = static_cast<size_t>(n) * C;
  double* U = c.alloc<double>(blk);
  double* Y = c.alloc<double>(blk);
  double* B = c.alloc<double>(blk);
  double* Phi = c.alloc<double>(blk);
  int32_t sweeps_max = 0;
  for (int32_t s0 = 0; s0 < ns; s0 += C) {
    const int cnt_s = std::min(C, ns - s0);
    const int32_t* srcc = src + s0;
    SBHA_CUDA(cudaMemsetAsync(U, 0, sizeof(double) * blk, c.stream));
    int32_t sweeps = 0;
    bool done = false;
    while (!done) {
      if (sweeps >= kMaxSweeps) {
        rep.converged = false;
        break;
      }
      for (int k = 0; k < kSweepsPerCheck; ++k, ++sweeps) {
        csr_block_spmm(c, n, g.nnz, g.rowptr, g.col, g.A, C, U, Y, 1.0);
        if (k == kSweepsPerCheck - 1) SBHA_CUDA(cudaMemsetAsync(chg, 0, sizeof(unsigned long long), c.stream));
        k_heat_sweep<<<grid_for(static_cast<int64_t>(blk), T), T, 0, c.stream>>>(n, nb, cnt_s, srcc, t, w, g.D, g.V,
                                                                                  Y, U, chg);
        c.launched("heat_sweep");
      }
      unsigned long long bits = 0;
      SBHA_CUDA(cudaMemcpyAsync(&bits, chg, sizeof(bits), cudaMemcpyDeviceToHost, c.stream));
      c.sync();
      double worst = 0.0;
      std::memcpy(&worst, &bits, sizeof(worst));
      if (!std::isfinite(worst)) SBHA_THROW(SBHA_ENOCONV, "the heat step diverged (a non-finite iterate)");
      done = worst <= kSweepTol;
    }
    sweeps_max = std::max(sweeps_max, sweeps);
    SBHA_CUDA(cudaMemsetAsync(B, 0, sizeof(double) * blk, c.stream));
    k_heat_div<<<grid_for(m.f * nb * BW, T), T, 0, c.stream>>>(m.f, n, nb, m.faces, m.xyz, U, B);
    c.launched("heat_div");
    k_heat_rhs<<<grid_for(static_cast<int64_t>(blk), T), T, 0, c.stream>>>(n, nb, B);
    c.launched("heat_rhs");
    SpdReport r = spd_block_solve(c, n, lnnz, lrowptr, lcol, lval, C, cnt_s, B, Phi, o);
    rep.iterations += r.iterations;
    rep.max_rel = std::max(rep.max_rel, r.max_rel);
    rep.converged = rep.converged && r.converged;
    k_heat_out<<<grid_for(static_cast<int64_t>(cnt_s) * n, T), T, 0, c.stream>>>(n, cnt_s, srcc, Phi,
                                                                                D + static_cast<int64_t>(s0) * n);
    c.launched("heat_out");
  }
  if (jacobi_iterations) *jacobi_iterations = sweeps_max;
  return rep;
}

}  // namespace sbha
