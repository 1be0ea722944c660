// Pattern construction and stabilised P1-P1 assembly on the device.
//
// Sec. 2.2 of arxiv 2310.10430: bilinear forms a (elasticity, with the lambda
// div-div term of sigma), b (coupling, -b -> B), c (K-weighted diffusion) and the
// stabilisation (beta/K) c(dp/dt, q) give per step
//   AA = [[A, B], [B^T, -(tau C + beta L)]],  A' = [[0, 0], [B^T, -beta L]]
// (Eq. fullysystem; L is the K-free Laplacian so that (beta/K_e) C_e = beta L_e on
// every element). DOFs are node-interleaved (3 v + f); the CSR pattern is the full
// element-coupling pattern: node v couples to itself and to its six grid
// neighbours (i+-1, j), (i, j+-1), (i+1, j+1), (i-1, j-1) of the "/"-split grid,
// each coupling a dense 3x3 block.
//
// Assembly is element-parallel in 8 colours (cell parity in x, in y, lower/upper
// triangle); triangles of one colour share no node, so the scatter needs no
// atomics and the summation order of every entry is fixed (colour 0..7).
#include "common.cuh"

#include <cmath>

namespace biot {

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// Sorted neighbour list of node v (self included); returns the count (<= 7).
__device__ __forceinline__ int node_neighbours(int n, int v, int* out) {
  const int nx = n + 1;
  const int i = v % nx, j = v / nx;
  int c = 0;
  if (i > 0 && j > 0) out[c++] = v - nx - 1;
  if (j > 0) out[c++] = v - nx;
  if (i > 0) out[c++] = v - 1;
  out[c++] = v;
  if (i < n) out[c++] = v + 1;
  if (j < n) out[c++] = v + nx;
  if (i < n && j < n) out[c++] = v + nx + 1;
  return c;
}

__global__ void k_degree(int n, int nn, int32_t* deg) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nn) return;
  int tmp[7];
  deg[v] = node_neighbours(n, v, tmp);
}

// Single-block exclusive scan: out[k] = sum_{m<k} in[m], out[N] = total.
__global__ void k_scan(const int32_t* __restrict__ in, int32_t* __restrict__ out, int N) {
  __shared__ int32_t s[1024];
  const int t = threadIdx.x;
  const int chunk = (N + 1023) / 1024;
  const int b = min(N, t * chunk), e = min(N, b + chunk);
  int32_t sum = 0;
  for (int k = b; k < e; ++k) sum += in[k];
  s[t] = sum;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    int32_t add = (t >= off) ? s[t - off] : 0;
    __syncthreads();
    s[t] += add;
    __syncthreads();
  }
  int32_t run = s[t] - sum;  // exclusive prefix of this chunk
  for (int k = b; k < e; ++k) {
    out[k] = run;
    run += in[k];
  }
  if (t == 1023) out[N] = s[1023];
}

__global__ void k_fill_pattern(int n, int nn, const int32_t* __restrict__ nodeptr, int32_t* __restrict__ nbr,
                               int32_t* __restrict__ rowptr, int32_t* __restrict__ col) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nn) return;
  int nb[7];
  const int deg = node_neighbours(n, v, nb);
  const int32_t np = nodeptr[v];
  for (int k = 0; k < deg; ++k) nbr[np + k] = nb[k];
  for (int f = 0; f < 3; ++f) {
    const int32_t rp = 9 * np + 3 * deg * f;
    rowptr[3 * v + f] = rp;
    for (int k = 0; k < deg; ++k)
      for (int g = 0; g < 3; ++g) col[rp + 3 * k + g] = 3 * nb[k] + g;
  }
  if (v == nn - 1) rowptr[3 * nn] = 9 * nodeptr[nn];
}

struct Material {
  double lam, mu, alpha, tau, beta;
};

// Vertices of triangle t (0 lower, 1 upper) of cell (i, j), counter-clockwise.
__device__ __forceinline__ void tri_vertices(int n, int i, int j, int t, int* vt) {
  const int nx = n + 1;
  const int v00 = j * nx + i, v10 = v00 + 1, v01 = v00 + nx, v11 = v01 + 1;
  vt[0] = v00;
  vt[1] = t == 0 ? v10 : v11;
  vt[2] = t == 0 ? v11 : v01;
}

// Area and constant gradients of the P1 basis on a triangle.
__device__ __forceinline__ void p1_grads(const double* x, const double* y, double& area, double* gx, double* gy) {
  const double det = (x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]);
  area = 0.5 * det;
  const double inv = 1.0 / det;
  for (int a = 0; a < 3; ++a) {
    const int b = (a + 1) % 3, c = (a + 2) % 3;
    gx[a] = (y[b] - y[c]) * inv;
    gy[a] = (x[c] - x[b]) * inv;
  }
}

__device__ __forceinline__ int find_slot(const int32_t* __restrict__ nbr, int32_t lo, int32_t hi, int m) {
  for (int32_t k = lo; k < hi; ++k)
    if (nbr[k] == m) return (int)(k - lo);
  return -1;
}

__device__ __forceinline__ void cell_of_colour(int n, int colour, int idx, int& i, int& j, int& t, bool& ok) {
  const int ci = colour & 1, cj = (colour >> 1) & 1;
  t = colour >> 2;
  const int ncx = (n - ci + 1) / 2, ncy = (n - cj + 1) / 2;
  ok = idx < ncx * ncy;
  i = ci + 2 * (idx % max(ncx, 1));
  j = cj + 2 * (idx / max(ncx, 1));
}

__global__ void k_assemble(int n, double hx, double hy, int colour, Material m, const double* __restrict__ kappa,
                           const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
                           const int32_t* __restrict__ rowptr, double* __restrict__ val, double* __restrict__ apval) {
  int i, j, t;
  bool ok;
  cell_of_colour(n, colour, blockIdx.x * blockDim.x + threadIdx.x, i, j, t, ok);
  if (!ok) return;
  int vt[3];
  tri_vertices(n, i, j, t, vt);
  const int nx = n + 1;
  double x[3], y[3];
  for (int a = 0; a < 3; ++a) {
    x[a] = (double)(vt[a] % nx) * hx;
    y[a] = (double)(vt[a] / nx) * hy;
  }
  double area, gx[3], gy[3];
  p1_grads(x, y, area, gx, gy);
  const double ke = kappa[2 * (j * n + i) + t];
  const double l2m = m.lam + 2.0 * m.mu;
  const double bc = -m.alpha * area / 3.0;
  for (int a = 0; a < 3; ++a) {
    const int va = vt[a];
    const int32_t np = nodeptr[va], ne = nodeptr[va + 1];
    const int32_t r0 = rowptr[3 * va], r1 = rowptr[3 * va + 1], r2 = rowptr[3 * va + 2];
    for (int b = 0; b < 3; ++b) {
      const int k = find_slot(nbr, np, ne, vt[b]);
      if (k < 0) continue;  // unreachable: triangle vertices are grid neighbours
      const double kxx = area * (l2m * gx[a] * gx[b] + m.mu * gy[a] * gy[b]);
      const double kxy = area * (m.lam * gx[a] * gy[b] + m.mu * gy[a] * gx[b]);
      const double kyx = area * (m.lam * gy[a] * gx[b] + m.mu * gx[a] * gy[b]);
      const double kyy = area * (l2m * gy[a] * gy[b] + m.mu * gx[a] * gx[b]);
      const double lab = area * (gx[a] * gx[b] + gy[a] * gy[b]);
      // u_x row of node a: (u_x, u_y, p) of node b
      val[r0 + 3 * k + 0] += kxx;
      val[r0 + 3 * k + 1] += kxy;
      val[r0 + 3 * k + 2] += bc * gx[a];          // B[(a,x), b]
      val[r1 + 3 * k + 0] += kyx;
      val[r1 + 3 * k + 1] += kyy;
      val[r1 + 3 * k + 2] += bc * gy[a];          // B[(a,y), b]
      // p row of node a: B^T[a, (b,x)] = B[(b,x), a], B^T[a, (b,y)], then -(tau C + beta L)
      val[r2 + 3 * k + 0] += bc * gx[b];
      val[r2 + 3 * k + 1] += bc * gy[b];
      val[r2 + 3 * k + 2] += -(m.tau * ke * lab + m.beta * lab);
      apval[np + k] += -m.beta * lab;
    }
  }
}

// Dirichlet DOFs of the four boundary-condition families.
__global__ void k_dirichlet_mask(int n, int problem, uint8_t* __restrict__ dmask) {
  const int nn = (n + 1) * (n + 1);
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nn) return;
  const int nx = n + 1, i = v % nx, j = v / nx;
  uint8_t m0 = 0, m1 = 0, m2 = 0;
  if (problem == BIOT_TERZAGHI) {
    if (j == 0) m0 = m1 = 1;            // fixed bottom
    if (i == 0 || i == n) m0 = 1;       // roller sides
    if (j == n) m2 = 1;                 // drained top
  } else if (problem == BIOT_BARRY_MERCER) {
    m0 = (j == 0 || j == n) ? 1 : 0;    // tangential u_x on the horizontal sides
    m1 = (i == 0 || i == n) ? 1 : 0;    // tangential u_y on the vertical sides
    m2 = (i == 0 || i == n || j == 0 || j == n) ? 1 : 0;  // drained everywhere
  } else if (problem == BIOT_MANDEL) {
    m0 = i == 0 ? 1 : 0;                // symmetry plane x = 0
    m1 = j == 0 ? 1 : 0;                // symmetry plane y = 0
    m2 = i == n ? 1 : 0;                // drained x = a
  } else {
    const bool bnd = (i == 0 || i == n || j == 0 || j == n);
    m0 = m1 = m2 = bnd ? 1 : 0;
  }
  dmask[3 * v] = m0;
  dmask[3 * v + 1] = m1;
  dmask[3 * v + 2] = m2;
}

// Spatial factor of the manufactured solution, cos(3 pi x) cos(3 pi y).
__device__ __forceinline__ double mms_phi(double x, double y) { return cos(3.0 * kPi * x) * cos(3.0 * kPi * y); }

// Manufactured sources split in time (Sec. 4.1 solution; sources from the PDE):
//   f_d = cos t * Sd(x),  g = sin t * G1(x) + cos t * G2(x).
__device__ __forceinline__ void mms_spatial(double x, double y, double lam, double mu, double alpha, double K,
                                            double& s1, double& s2, double& g1, double& g2) {
  const double k = 3.0 * kPi;
  const double cx = cos(k * x), sx = sin(k * x), cy = cos(k * y), sy = sin(k * y);
  const double common = k * k * ((lam + 3.0 * mu) * cx * cy - (lam + mu) * sx * sy);
  s1 = common - alpha * k * sx * cy;
  s2 = common - alpha * k * cx * sy;
  g1 = alpha * k * (sx * cy + cx * sy);
  g2 = 2.0 * K * k * k * cx * cy;
}

// Element loads by the 3-point edge-midpoint rule: phi_a = 1/2 at the midpoints
// of the two edges through vertex a. Output per node: su (3 v + d), sg1, sg2.
__global__ void k_mms_loads(int n, double hx, double hy, int colour, double lam, double mu, double alpha, double K,
                            double* __restrict__ su, double* __restrict__ sg1, double* __restrict__ sg2) {
  int i, j, t;
  bool ok;
  cell_of_colour(n, colour, blockIdx.x * blockDim.x + threadIdx.x, i, j, t, ok);
  if (!ok) return;
  int vt[3];
  tri_vertices(n, i, j, t, vt);
  const int nx = n + 1;
  double x[3], y[3];
  for (int a = 0; a < 3; ++a) {
    x[a] = (double)(vt[a] % nx) * hx;
    y[a] = (double)(vt[a] / nx) * hy;
  }
  const double area = 0.5 * ((x[1] - x[0]) * (y[2] - y[0]) - (x[2] - x[0]) * (y[1] - y[0]));
  double q[3][4];  // midpoint values of (s1, s2, g1, g2) for edges (0,1), (1,2), (2,0)
  for (int e = 0; e < 3; ++e) {
    const int a = e, b = (e + 1) % 3;
    mms_spatial(0.5 * (x[a] + x[b]), 0.5 * (y[a] + y[b]), lam, mu, alpha, K, q[e][0], q[e][1], q[e][2], q[e][3]);
  }
  for (int a = 0; a < 3; ++a) {
    const int e1 = a, e2 = (a + 2) % 3;  // edges (a, a+1) and (a-1, a)
    double w[4];
    for (int c = 0; c < 4; ++c) w[c] = area / 3.0 * 0.5 * (q[e1][c] + q[e2][c]);
    const int v = vt[a];
    su[3 * v] += w[0];
    su[3 * v + 1] += w[1];
    sg1[v] += w[2];
    sg2[v] += w[3];
  }
}

// Lifting vectors of the manufactured case (g_D(t) = cos t * phi on Dirichlet DOFs):
//   l1 = AA_full[:, D] phi,  l2 = A'_full[:, D] phi  (computed before elimination).
__global__ void k_lifting(int n, int n_dof, double hx, double hy, const int32_t* __restrict__ rowptr,
                          const int32_t* __restrict__ col, const double* __restrict__ val,
                          const int32_t* __restrict__ nodeptr, const double* __restrict__ apval,
                          const uint8_t* __restrict__ dmask, double* __restrict__ l1, double* __restrict__ l2) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_dof) return;
  const int nx = n + 1;
  double s1 = 0.0, s2 = 0.0;
  const int v = r / 3, f = r % 3;
  for (int32_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
    const int c = col[e];
    if (!dmask[c]) continue;
    const int m = c / 3;
    const double ph = mms_phi((double)(m % nx) * hx, (double)(m / nx) * hy);
    s1 += val[e] * ph;
    if (f == 2) {
      const int g = c % 3;
      if (g < 2) {
        s2 += val[e] * ph;  // A' shares B^T with AA
      } else {
        const int k = (int)((e - rowptr[r]) / 3);
        s2 += apval[nodeptr[v] + k] * ph;
      }
    }
  }
  l1[r] = s1;
  l2[r] = s2;
}

// cos(t_k), sin(omega t_k) for k = 0..n_t (omega = 1: manufactured case; Barry & Mercer: beta).
__global__ void k_time_tables(int n_t, double tau, double omega, double* __restrict__ tc, double* __restrict__ ts) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > n_t) return;
  const double t = (double)k * tau;
  tc[k] = cos(t);
  ts[k] = sin(omega * t);
}

// Barry & Mercer's point source: the P1 basis of the triangle holding the point, evaluated there
// (the load of a Dirac delta), on its three vertices; amp: the source's amplitude (g = amp sin).
struct PointSource {
  int v[3];
  double w[3];
  double amp;
};

// F[r][k] for k = 0..n_t (column 0 zero). Terzaghi: constant traction on u_y of
// the top nodes for t_k >= tau. Manufactured case: loads, -tau G and lifting. Barry & Mercer:
// -tau G on the pressure rows of the source triangle's vertices, G = w_v amp sin(beta t_k).
__global__ void k_rhs(int n, int n_dof, int n_t, int ldx, int problem, double hx, double hy, double tau, double load,
                      const uint8_t* __restrict__ dmask, const double* __restrict__ su, const double* __restrict__ sg1,
                      const double* __restrict__ sg2, const double* __restrict__ l1, const double* __restrict__ l2,
                      const double* __restrict__ tc, const double* __restrict__ ts, PointSource ps,
                      double* __restrict__ F) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_dof) return;
  const int nx = n + 1, v = r / 3, f = r % 3, i = v % nx, j = v / nx;
  double* Fr = F + (size_t)r * ldx;
  Fr[0] = 0.0;
  if (problem == BIOT_TERZAGHI || problem == BIOT_MANDEL) {  // `load`: the top traction's magnitude
    double val = 0.0;
    if (f == 1 && j == n && !dmask[r]) val = -load * 0.5 * hx * ((i > 0 ? 1.0 : 0.0) + (i < n ? 1.0 : 0.0));
    for (int k = 1; k <= n_t; ++k) Fr[k] = val;  // Dirichlet data are zero
    return;
  }
  if (problem == BIOT_BARRY_MERCER) {
    double w = 0.0;
    if (f == 2 && !dmask[r])
      for (int a = 0; a < 3; ++a)
        if (ps.v[a] == v) w += ps.w[a];
    for (int k = 1; k <= n_t; ++k) Fr[k] = -tau * (w * ps.amp * ts[k]);
    return;
  }
  if (dmask[r]) {
    const double ph = mms_phi((double)i * hx, (double)j * hy);
    const double sgn = (f == 2) ? -1.0 : 1.0;
    for (int k = 1; k <= n_t; ++k) Fr[k] = sgn * tc[k] * ph;
    return;
  }
  for (int k = 1; k <= n_t; ++k) {
    double load_k = (f < 2) ? tc[k] * su[r] : -tau * (ts[k] * sg1[v] + tc[k] * sg2[v]);
    Fr[k] = load_k - tc[k] * l1[r] + tc[k - 1] * l2[r];
  }
}

// Mandel's undrained initial state (Sec. 4.3): u = (ux_x x, uy_y y), p = p0.
struct Undrained {
  double ux_x, uy_y, p0;
};

// Initial state x0 (column 0) and the zero initial guess X^{n,0} = 0 (Alg. 3).
__global__ void k_init_state(int n, int n_dof, int n_t, int ldx, int problem, double hx, double hy, Undrained ud,
                             double* __restrict__ X) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_dof) return;
  double* Xr = X + (size_t)r * ldx;
  double x0 = 0.0;
  if (problem == BIOT_MMS_TRIG) {
    const int nx = n + 1, v = r / 3;
    x0 = mms_phi((double)(v % nx) * hx, (double)(v / nx) * hy);
  } else if (problem == BIOT_MANDEL) {
    const int nx = n + 1, v = r / 3, f = r % 3;
    x0 = f == 0 ? ud.ux_x * ((double)(v % nx) * hx) : f == 1 ? ud.uy_y * ((double)(v / nx) * hy) : ud.p0;
  }
  Xr[0] = x0;
  for (int k = 1; k < ldx; ++k) Xr[k] = 0.0;
}

// Mandel's rigid plate (reading of Sec. 4.3): the penalty kp (u_y(i+1) - u_y(i))^2 / 2 over
// consecutive top nodes, added to the u_y row of every top node (one thread per node: its
// diagonal gets kp per top neighbour, each top neighbour's entry -kp; no two threads share a row).
__global__ void k_mandel_penalty(int n, double kp, const int32_t* __restrict__ nodeptr,
                                 const int32_t* __restrict__ nbr, const int32_t* __restrict__ rowptr,
                                 double* __restrict__ val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  const int v = n * (n + 1) + i;
  const int32_t np = nodeptr[v];
  const int deg = nodeptr[v + 1] - np;
  const int32_t r1 = rowptr[3 * v] + 3 * deg;  // the u_y row of node v
  for (int k = 0; k < deg; ++k) {
    const int m = nbr[np + k];
    double add = 0.0;
    if (m == v) add = kp * ((i > 0 ? 1.0 : 0.0) + (i < n ? 1.0 : 0.0));
    else if ((m == v - 1 && i > 0) || (m == v + 1 && i < n)) add = -kp;
    val[r1 + 3 * k + 1] += add;
  }
}

// Symmetric elimination: zero Dirichlet rows and columns (pattern kept), diagonal
// +1 (u) / -1 (p); the same rows and columns of A'_pp are zeroed.
__global__ void k_eliminate(int n_dof, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const int32_t* __restrict__ nodeptr, const int32_t* __restrict__ nbr,
                            const uint8_t* __restrict__ dmask, double* __restrict__ val, double* __restrict__ apval) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_dof) return;
  const bool dr = dmask[r];
  for (int32_t e = rowptr[r]; e < rowptr[r + 1]; ++e) {
    const int c = col[e];
    if (dr)
      val[e] = (c == r) ? ((r % 3 == 2) ? -1.0 : 1.0) : 0.0;
    else if (dmask[c])
      val[e] = 0.0;
  }
  if (r % 3 == 2) {
    const int v = r / 3;
    for (int32_t k = nodeptr[v]; k < nodeptr[v + 1]; ++k)
      if (dr || dmask[3 * nbr[k] + 2]) apval[k] = 0.0;
  }
}

__global__ void k_dscale(int n_dof, const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                         const double* __restrict__ val, double* __restrict__ dsc, double* __restrict__ dsq) {
  int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_dof) return;
  double d = 0.0;
  for (int32_t e = rowptr[r]; e < rowptr[r + 1]; ++e)
    if (col[e] == r) d = val[e];
  dsc[r] = 1.0 / sqrt(fabs(d));
  dsq[r] = sqrt(fabs(d));
}

}  // namespace

biot_status build_pattern(biot_ctx* ctx) {
  const int nn = ctx->n_nodes;
  int32_t* deg = nullptr;
  BIOT_TRY(dalloc(ctx, (void**)&deg, sizeof(int32_t) * nn));
  BIOT_TRY(dalloc(ctx, (void**)&ctx->nodeptr, sizeof(int32_t) * (nn + 1)));
  BIOT_TRY(dalloc(ctx, (void**)&ctx->nbr, sizeof(int32_t) * ctx->n_pairs));
  BIOT_TRY(dalloc(ctx, (void**)&ctx->rowptr, sizeof(int32_t) * (ctx->n_dof + 1)));
  BIOT_TRY(dalloc(ctx, (void**)&ctx->col, sizeof(int32_t) * ctx->nnz));
  BIOT_LAUNCH(k_degree, div_up(nn, 256), 256, 0, ctx->stream, ctx->n, nn, deg);
  BIOT_LAUNCH(k_scan, 1, 1024, 0, ctx->stream, deg, ctx->nodeptr, nn);
  BIOT_LAUNCH(k_fill_pattern, div_up(nn, 256), 256, 0, ctx->stream, ctx->n, nn, ctx->nodeptr, ctx->nbr, ctx->rowptr,
              ctx->col);
  BIOT_CU(ctx, cudaGetLastError());
  return BIOT_OK;
}

// k_p / (lambda + 2 mu) of Mandel's rigid-plate penalty (reading of Sec. 4.3)
constexpr double kMandelPenalty = 1e4;

biot_status assemble_system(biot_ctx* ctx) {
  const biot_params& p = ctx->prm;
  const int n = ctx->n, nn = ctx->n_nodes, nd = ctx->n_dof;
  const double hx = ctx->Lx / n, hy = ctx->Ly / n;
  cudaStream_t s = ctx->stream;
  const double lam = p.E * p.nu / ((1.0 + p.nu) * (1.0 - 2.0 * p.nu));
  const double mu = p.E / (2.0 * (1.0 + p.nu));
  const double h = (ctx->Lx > ctx->Ly ? ctx->Lx : ctx->Ly) / n;
  double beta = 0.0;
  if (p.beta_mode == BIOT_BETA_H2) beta = h * h / (4.0 * (lam + 2.0 * mu));
  if (p.beta_mode == BIOT_BETA_H) beta = h / (4.0 * (lam + 2.0 * mu));
  if (ctx->beta_force >= 0.0) beta = ctx->beta_force;  // a multigrid level keeps the fine beta
  ctx->beta = beta;
  Material m{lam, mu, p.alpha, p.tau, beta};

  BIOT_CU(ctx, cudaMemsetAsync(ctx->val, 0, sizeof(double) * ctx->nnz, s));
  BIOT_CU(ctx, cudaMemsetAsync(ctx->apval, 0, sizeof(double) * ctx->n_pairs, s));
  const int cells_per_colour = ((n + 1) / 2) * ((n + 1) / 2);
  for (int colour = 0; colour < 8; ++colour)
    BIOT_LAUNCH(k_assemble, div_up(cells_per_colour, 128), 128, 0, s, n, hx, hy, colour, m, ctx->kappa, ctx->nodeptr,
                ctx->nbr, ctx->rowptr, ctx->val, ctx->apval);
  BIOT_LAUNCH(k_dirichlet_mask, div_up(nn, 256), 256, 0, s, n, p.problem, ctx->dmask);
  Undrained ud{0.0, 0.0, 0.0};
  double tload = p.load;
  if (p.problem == BIOT_MANDEL) {
    BIOT_LAUNCH(k_mandel_penalty, div_up(n + 1, 128), 128, 0, s, n, kMandelPenalty * (lam + 2.0 * mu), ctx->nodeptr,
                ctx->nbr, ctx->rowptr, ctx->val);
    // Skempton B = 1 (alpha = 1, no storage), nu_u = (3 nu + B (1 - 2 nu)) / (3 - B (1 - 2 nu)); the
    // force F = load on the quarter's top as the traction F / a
    const double B = 1.0, nu = p.nu, a = ctx->Lx;
    const double nu_u = (3.0 * nu + B * (1.0 - 2.0 * nu)) / (3.0 - B * (1.0 - 2.0 * nu));
    ud.ux_x = p.load * nu_u / (2.0 * mu * a);
    ud.uy_y = -p.load * (1.0 - nu_u) / (2.0 * mu * a);
    ud.p0 = p.load * B * (1.0 + nu_u) / (3.0 * a);
    tload = p.load / a;
  }

  // right-hand sides (needs the matrices before elimination for the lifting)
  double *su = nullptr, *sg = nullptr, *lift = nullptr, *tt = nullptr;
  const size_t tmp_doubles = (size_t)nd + 2 * (size_t)nn + 2 * (size_t)nd + 2 * (size_t)(p.n_t + 1);
  double* tmp = nullptr;
  BIOT_CU(ctx, cudaMallocAsync((void**)&tmp, sizeof(double) * tmp_doubles, s));
  su = tmp;
  sg = su + nd;
  lift = sg + 2 * (size_t)nn;
  tt = lift + 2 * (size_t)nd;
  BIOT_CU(ctx, cudaMemsetAsync(tmp, 0, sizeof(double) * tmp_doubles, s));
  // Barry & Mercer: beta = (lambda + 2 mu) K / (a b), the source at (a/4, b/4)
  PointSource ps{{-1, -1, -1}, {0.0, 0.0, 0.0}, -0.5 * p.load};
  double omega = 1.0;
  if (p.problem == BIOT_BARRY_MERCER) {
    const double K = p.kappa_elem ? p.kappa_elem[0] : p.kappa_const;
    omega = (lam + 2.0 * mu) * K / (ctx->Lx * ctx->Ly);
    // cell of the point and its local coordinates; the "/" diagonal splits the cell into the
    // lower triangle (xi >= eta) and the upper one
    const double px = ctx->Lx / 4.0 / hx, py = ctx->Ly / 4.0 / hy;
    const int ci = std::min((int)std::floor(px), n - 1), cj = std::min((int)std::floor(py), n - 1);
    const double xi = px - ci, eta = py - cj;
    const int nx = n + 1, v00 = cj * nx + ci, v10 = v00 + 1, v11 = v00 + nx + 1, v01 = v00 + nx;
    if (xi >= eta) ps = {{v00, v10, v11}, {1.0 - xi, xi - eta, eta}, ps.amp};
    else ps = {{v00, v11, v01}, {1.0 - eta, xi, eta - xi}, ps.amp};
  }
  BIOT_LAUNCH(k_time_tables, div_up(p.n_t + 1, 256), 256, 0, s, p.n_t, p.tau, omega, tt, tt + p.n_t + 1);
  if (p.problem == BIOT_MMS_TRIG) {
    // the manufactured case assumes a constant K (first element's value)
    double K = p.kappa_const;
    if (p.kappa_elem) K = p.kappa_elem[0];
    for (int colour = 0; colour < 8; ++colour)
      BIOT_LAUNCH(k_mms_loads, div_up(cells_per_colour, 128), 128, 0, s, n, hx, hy, colour, lam, mu, p.alpha, K, su, sg,
                  sg + nn);
    BIOT_LAUNCH(k_lifting, div_up(nd, 256), 256, 0, s, n, nd, hx, hy, ctx->rowptr, ctx->col, ctx->val, ctx->nodeptr,
                ctx->apval, ctx->dmask, lift, lift + nd);
  }
  BIOT_LAUNCH(k_rhs, div_up(nd, 128), 128, 0, s, n, nd, p.n_t, ctx->ldx, p.problem, hx, hy, p.tau, tload, ctx->dmask,
              su, sg, sg + nn, lift, lift + nd, tt, tt + p.n_t + 1, ps, ctx->F);
  BIOT_LAUNCH(k_init_state, div_up(nd, 128), 128, 0, s, n, nd, p.n_t, ctx->ldx, p.problem, hx, hy, ud, ctx->X);
  BIOT_LAUNCH(k_eliminate, div_up(nd, 256), 256, 0, s, nd, ctx->rowptr, ctx->col, ctx->nodeptr, ctx->nbr, ctx->dmask,
              ctx->val, ctx->apval);
  BIOT_LAUNCH(k_dscale, div_up(nd, 256), 256, 0, s, nd, ctx->rowptr, ctx->col, ctx->val, ctx->dsc, ctx->dsq);
  BIOT_CU(ctx, cudaGetLastError());
  BIOT_CU(ctx, cudaFreeAsync(tmp, s));
  return BIOT_OK;
}

}  // namespace biot
