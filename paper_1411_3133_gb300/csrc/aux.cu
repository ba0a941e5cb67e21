// Initialisation, macroscopic fields, state conversion and the observables
// reduction (Sec. II initial state and moments; Sec. III-IV Dean number,
// mean velocity and mean vorticity).
#include "kernels.cuh"
#include "launch.h"

namespace lbgm {

namespace {

uint32_t blocks_for(const Dims& d, int threads) {
  const uint32_t total = uint32_t(d.batch) * uint32_t(d.ncell);
  return (total + threads - 1) / threads;
}

template <typename S, typename Real>
cudaError_t macros_t(int K, const S* fin, double* rho, double* u, const Dims& d, cudaStream_t s) {
  const uint32_t nb = blocks_for(d, 256);
  switch (K) {
    case KFLAT: k_macros<S, Real, KFLAT><<<nb, 256, 0, s>>>(fin, rho, u, d); break;
    case KCYL: k_macros<S, Real, KCYL><<<nb, 256, 0, s>>>(fin, rho, u, d); break;
    case KELL: k_macros<S, Real, KELL><<<nb, 256, 0, s>>>(fin, rho, u, d); break;
    case KELT:
      if constexpr (!Codec<S, Real>::uses_ref) {  // FP64 / FP32 storage only
        k_macros<S, Real, KELT><<<nb, 256, 0, s>>>(fin, rho, u, d);
        break;
      }
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename S, typename Real>
cudaError_t init_t(int K, S* f, const GeoDev<Real>& geo, const double* sqrtg, const double* base,
                   const InitInst* ini, const double* rho_in, const double* u_in, const Dims& d,
                   cudaStream_t s) {
  const uint32_t nb = blocks_for(d, 256);
  switch (K) {
    case KFLAT: k_init<S, Real, KFLAT><<<nb, 256, 0, s>>>(f, geo, sqrtg, base, ini, rho_in, u_in, d); break;
    case KCYL: k_init<S, Real, KCYL><<<nb, 256, 0, s>>>(f, geo, sqrtg, base, ini, rho_in, u_in, d); break;
    case KELL: k_init<S, Real, KELL><<<nb, 256, 0, s>>>(f, geo, sqrtg, base, ini, rho_in, u_in, d); break;
    case KELT:
      if constexpr (!Codec<S, Real>::uses_ref) {  // FP64 / FP32 storage only
        k_init<S, Real, KELT><<<nb, 256, 0, s>>>(f, geo, sqrtg, base, ini, rho_in, u_in, d);
        break;
      }
      return cudaErrorInvalidValue;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// weights by population index, for the element-wise conversions
__constant__ double c_weight[Q];

// stored value <-> f_l (2-byte formats: f = w s + r, Codec)
__device__ __forceinline__ double to_f(double v, double, double) { return v; }
__device__ __forceinline__ double to_f(float v, double, double) { return v; }
__device__ __forceinline__ double to_f(__half v, double w, double r) { return w * double(__half2float(v)) + r; }
__device__ __forceinline__ double to_f(__nv_bfloat16 v, double w, double r) {
  return w * double(__bfloat162float(v)) + r;
}
__device__ __forceinline__ void from_f(double& o, double f, double, double) { o = f; }
__device__ __forceinline__ void from_f(float& o, double f, double, double) { o = float(f); }
__device__ __forceinline__ void from_f(__half& o, double f, double w, double r) { o = __double2half((f - r) / w); }
__device__ __forceinline__ void from_f(__nv_bfloat16& o, double f, double w, double r) {
  o = __double2bfloat16((f - r) / w);
}

// state (documented population layout) <-> FP64 populations
template <typename S>
__global__ void k_convert(S* state, double* dbl, size_t n, Dims d, int to_double) {
  const size_t N = size_t(d.ncell), layer = size_t(d.nt) * size_t(d.n3);
  const size_t nrows = size_t(d.nr) * size_t(d.geo_rows3);
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < n;
       i += size_t(gridDim.x) * blockDim.x) {
    const size_t bl = i / N;  // b * Q + l
    const double w = c_weight[bl % Q];
    double r = 0.0;
    if (d.ref) {  // the reference table's layout of ref_index
      const size_t cell = i - bl * N, b = bl / Q, l = bl % Q;
      const size_t ir = cell / layer;
      const float* rb = d.ref + b * Q * nrows;
      r = d.geo_rows3 > 1 ? double(rb[l * nrows + ir * size_t(d.geo_rows3) + cell % size_t(d.n3)])
                          : double(rb[ir * Q + l]);
    }
    if (to_double)
      dbl[i] = to_f(state[i], w, r);
    else
      from_f(state[i], dbl[i], w, r);
  }
}

// Equilibrium walls: the wall nodes' velocity is the Dirichlet value 0 in
// every observable (their streamed moments are replaced in the collision).
__device__ __forceinline__ bool eq_wall_node(const Dims& d, int ir, int i3) {
  return d.wall_eq && (ir == 0 || ir == d.nr - 1 || (!d.periodic3 && (i3 == 0 || i3 == d.n3 - 1)));
}

// mean of u^r along x3 for every (instance, i_r, i_theta) row
__global__ void k_rowmean(const double* __restrict__ u, double* __restrict__ rowmean, Dims d) {
  const int rows_per = d.nr * d.nt;
  const int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= d.batch * rows_per) return;
  const int b = row / rows_per;
  const int rr = row - b * rows_per;
  const int ir = rr / d.nt;
  const double* ur = u + size_t(b) * 3 * d.ncell + size_t(rr) * d.n3;
  double s = 0.0;
  for (int i = 0; i < d.n3; ++i) s += eq_wall_node(d, ir, i) ? 0.0 : ur[i];
  rowmean[row] = s / d.n3;
}

// derivative along an axis from the values at offsets -2 .. +2 (u2m, um, u0,
// up, u2p); the bounce-back wall version uses u = 0 half a node outside the
// first and last node, the equilibrium-wall version second-order one-sided
// differences at the wall nodes (whose value is 0).
__device__ __forceinline__ double d_axis(double u2m, double um, double u0, double up, double u2p, int i, int n,
                                         bool walled, bool eqw) {
  if (!walled) return 0.5 * (up - um);
  if (n == 1) return 0.0;
  if (eqw) {
    if (i == 0) return 0.5 * (-3.0 * u0 + 4.0 * up - u2p);
    if (i == n - 1) return 0.5 * (3.0 * u0 - 4.0 * um + u2m);
    return 0.5 * (up - um);
  }
  if (i == 0) return u0 + up / 3.0;
  if (i == n - 1) return -(u0 + um / 3.0);
  return 0.5 * (up - um);
}

constexpr int DIAG_THREADS = 256;

__device__ __forceinline__ void block_reduce(double (&a)[DIAG_NQ], double* sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < DIAG_NQ; ++q) {
    double v = a[q];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double w = __shfl_down_sync(0xffffffffu, v, o);
      v = (q == 7) ? fmax(v, w) : v + w;
    }
    if (lane == 0) sh[warp * DIAG_NQ + q] = v;
  }
  __syncthreads();
  if (threadIdx.x < DIAG_NQ) {
    const int q = threadIdx.x;
    double v = sh[q];
    for (int w = 1; w < DIAG_THREADS / 32; ++w)
      v = (q == 7) ? fmax(v, sh[w * DIAG_NQ + q]) : v + sh[w * DIAG_NQ + q];
    a[q] = v;  // valid in thread q only
  }
}

// Per-block partial sums of one instance (blockIdx.y), in a fixed order.
//   0 rho'   1 rho' g   2 sqrt(g_thth) u^theta wA   3 wA   4 |omega| wOmega
//   5 (u^r)^2   6 (u^r - row mean)^2   7 max |u|   8 non-finite nodes
__global__ void __launch_bounds__(DIAG_THREADS)
    k_diag_partial(const double* __restrict__ rho, const double* __restrict__ u,
                   const double* __restrict__ rowmean, const double* __restrict__ geo64, Dims d,
                   double* __restrict__ partial, int nblk) {
  __shared__ double sh[(DIAG_THREADS / 32) * DIAG_NQ];
  const int b = blockIdx.y;
  const int N = d.ncell;
  const double* ur = u + size_t(b) * 3 * N;
  const double* ut = ur + N;
  const double* uz = ur + 2 * size_t(N);
  const double* rb = rho + size_t(b) * N;
  double a[DIAG_NQ];
#pragma unroll
  for (int q = 0; q < DIAG_NQ; ++q) a[q] = 0.0;
  const int plane = d.nt * d.n3;
  for (int c = blockIdx.x * DIAG_THREADS + threadIdx.x; c < N; c += nblk * DIAG_THREADS) {
    const int ir = c / plane;
    const int rem = c - ir * plane;
    const int it = rem / d.n3;
    const int i3 = rem - it * d.n3;
    const double* gr = geo64 + size_t(d.geo_theta ? c : ir * d.n3 + i3) * 4;
    const double sg = gr[0], sp = gr[1], wA = gr[2], wOm = gr[3];
    const double r = rb[c];
    const bool eqw = d.wall_eq != 0;
    // velocity component at node (jr, j3) of this theta plane: 0 on an
    // equilibrium wall node and outside the node range
    auto U = [&](const double* a, int jr, int j3) -> double {
      if (jr < 0 || jr >= d.nr || j3 < 0 || j3 >= d.n3 || eq_wall_node(d, jr, j3)) return 0.0;
      return a[(size_t(jr) * d.nt + it) * d.n3 + j3];
    };
    const double u0 = U(ur, ir, i3), u1 = U(ut, ir, i3), u2 = U(uz, ir, i3);
    // d_3 u^r
    double d3ur;
    if (d.periodic3) {
      const int jm = i3 == 0 ? d.n3 - 1 : i3 - 1, jp = i3 == d.n3 - 1 ? 0 : i3 + 1;
      d3ur = d_axis(0.0, U(ur, ir, jm), u0, U(ur, ir, jp), 0.0, i3, d.n3, false, eqw);
    } else {
      d3ur = d_axis(U(ur, ir, i3 - 2), U(ur, ir, i3 - 1), u0, U(ur, ir, i3 + 1), U(ur, ir, i3 + 2), i3, d.n3,
                    true, eqw);
    }
    // d_r u^3 (walls on r)
    const double drz = d_axis(U(uz, ir - 2, i3), U(uz, ir - 1, i3), u2, U(uz, ir + 1, i3), U(uz, ir + 2, i3), ir,
                              d.nr, true, eqw);
    const double fl = u0 - rowmean[(size_t(b) * d.nr + ir) * d.nt + it];
    a[0] += r;
    a[1] += sg * sg * r;
    a[2] += sp * u1 * wA;
    a[3] += wA;
    a[4] += fabs(d3ur - drz) * wOm;
    a[5] += u0 * u0;
    a[6] += fl * fl;
    a[7] = fmax(a[7], sqrt(u0 * u0 + u1 * u1 + u2 * u2));
    const bool fin = isfinite(r) && isfinite(u0) && isfinite(u1) && isfinite(u2);
    a[8] += fin ? 0.0 : 1.0;
  }
  block_reduce(a, sh);
  if (threadIdx.x < DIAG_NQ) partial[(size_t(b) * nblk + blockIdx.x) * DIAG_NQ + threadIdx.x] =
      a[threadIdx.x];
}

__global__ void __launch_bounds__(DIAG_THREADS)
    k_diag_final(const double* __restrict__ partial, int nblk, double* __restrict__ out) {
  __shared__ double sh[(DIAG_THREADS / 32) * DIAG_NQ];
  const int b = blockIdx.x;
  double a[DIAG_NQ];
#pragma unroll
  for (int q = 0; q < DIAG_NQ; ++q) a[q] = 0.0;
  for (int k = threadIdx.x; k < nblk; k += DIAG_THREADS) {
    const double* p = partial + (size_t(b) * nblk + k) * DIAG_NQ;
#pragma unroll
    for (int q = 0; q < DIAG_NQ; ++q) a[q] = (q == 7) ? fmax(a[q], p[q]) : a[q] + p[q];
  }
  block_reduce(a, sh);
  if (threadIdx.x < DIAG_NQ) out[size_t(b) * DIAG_NQ + threadIdx.x] = a[threadIdx.x];
}

}  // namespace

cudaError_t launch_macros(int prec, int K, const void* fin, double* rho, double* u, const Dims& d,
                          cudaStream_t s) {
  switch (prec) {
    case 0: return macros_t<double, double>(K, static_cast<const double*>(fin), rho, u, d, s);
    case 1: return macros_t<float, float>(K, static_cast<const float*>(fin), rho, u, d, s);
    case 2: return macros_t<__half, float>(K, static_cast<const __half*>(fin), rho, u, d, s);
    case 3: return macros_t<__nv_bfloat16, float>(K, static_cast<const __nv_bfloat16*>(fin), rho, u, d, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_init(int prec, int K, void* f, const void* geo, const double* sqrtg,
                        const double* base_uth, const InitInst* ini, const double* rho_in,
                        const double* u_in, const Dims& d, cudaStream_t s) {
  const GeoDev<float>& gf = *static_cast<const GeoDev<float>*>(geo);
  switch (prec) {
    case 0:
      return init_t<double, double>(K, static_cast<double*>(f), *static_cast<const GeoDev<double>*>(geo),
                                    sqrtg, base_uth, ini, rho_in, u_in, d, s);
    case 1: return init_t<float, float>(K, static_cast<float*>(f), gf, sqrtg, base_uth, ini, rho_in, u_in, d, s);
    case 2: return init_t<__half, float>(K, static_cast<__half*>(f), gf, sqrtg, base_uth, ini, rho_in, u_in, d, s);
    case 3:
      return init_t<__nv_bfloat16, float>(K, static_cast<__nv_bfloat16*>(f), gf, sqrtg, base_uth, ini, rho_in,
                                          u_in, d, s);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_convert(int prec, int to_double, void* state, double* dbl, size_t n, const Dims& d,
                           cudaStream_t s) {
  static bool weights_set = false;
  if (!weights_set) {
    double w[Q];
    for (int l = 0; l < Q; ++l) w[l] = weight(l);
    cudaError_t e = cudaMemcpyToSymbol(c_weight, w, sizeof(w));
    if (e != cudaSuccess) return e;
    weights_set = true;
  }
  const int threads = 256;
  const size_t want = (n + threads - 1) / threads;
  const int blocks = int(want < 152 * 16 ? (want ? want : 1) : 152 * 16);
  switch (prec) {
    case 0: k_convert<double><<<blocks, threads, 0, s>>>(static_cast<double*>(state), dbl, n, d, to_double); break;
    case 1: k_convert<float><<<blocks, threads, 0, s>>>(static_cast<float*>(state), dbl, n, d, to_double); break;
    case 2: k_convert<__half><<<blocks, threads, 0, s>>>(static_cast<__half*>(state), dbl, n, d, to_double); break;
    case 3:
      k_convert<__nv_bfloat16><<<blocks, threads, 0, s>>>(static_cast<__nv_bfloat16*>(state), dbl, n, d,
                                                          to_double);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// Per instance (blockIdx.y): max |u - u_prev| and max |u| over the nodes,
// then u_prev = u. Partial maxima per block, reduced by k_residual_final.
__global__ void __launch_bounds__(256) k_residual(const double* __restrict__ u, double* __restrict__ u_prev,
                                                  size_t per_inst, double* __restrict__ partial, int nblk) {
  __shared__ double sd[256], su[256];
  const size_t b = blockIdx.y;
  double md = 0.0, mu = 0.0;
  for (size_t i = blockIdx.x * size_t(blockDim.x) + threadIdx.x; i < per_inst; i += size_t(nblk) * blockDim.x) {
    const size_t k = b * per_inst + i;
    const double v = u[k];
    md = fmax(md, fabs(v - u_prev[k]));
    mu = fmax(mu, fabs(v));
    u_prev[k] = v;
  }
  sd[threadIdx.x] = md;
  su[threadIdx.x] = mu;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sd[threadIdx.x] = fmax(sd[threadIdx.x], sd[threadIdx.x + s]);
      su[threadIdx.x] = fmax(su[threadIdx.x], su[threadIdx.x + s]);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    partial[(b * nblk + blockIdx.x) * 2] = sd[0];
    partial[(b * nblk + blockIdx.x) * 2 + 1] = su[0];
  }
}

__global__ void k_residual_final(const double* __restrict__ partial, int nblk, int batch, double* __restrict__ out) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= batch) return;
  double md = 0.0, mu = 0.0;
  for (int i = 0; i < nblk; ++i) {
    md = fmax(md, partial[(size_t(b) * nblk + i) * 2]);
    mu = fmax(mu, partial[(size_t(b) * nblk + i) * 2 + 1]);
  }
  out[2 * b] = md;
  out[2 * b + 1] = mu;
}

cudaError_t launch_residual(const double* u, double* u_prev, const Dims& d, double* partial, int nblk,
                            double* out, cudaStream_t s) {
  const size_t per = size_t(3) * d.ncell;
  k_residual<<<dim3(nblk, d.batch), 256, 0, s>>>(u, u_prev, per, partial, nblk);
  k_residual_final<<<(d.batch + 255) / 256, 256, 0, s>>>(partial, nblk, d.batch, out);
  return cudaGetLastError();
}

// Row means of FP64 populations into the reference table (ref_index
// layout): one thread per (instance, row, population).
__global__ void k_ref_from_state(const double* __restrict__ dbl, float* __restrict__ ref, Dims d) {
  const size_t nrows = size_t(d.nr) * size_t(d.geo_rows3);
  const size_t t = blockIdx.x * size_t(blockDim.x) + threadIdx.x;
  if (t >= size_t(d.batch) * nrows * Q) return;
  const size_t l = t % Q, br = t / Q, b = br / nrows, row = br - b * nrows;
  const int ir = int(row / size_t(d.geo_rows3)), i3 = int(row - size_t(ir) * d.geo_rows3);
  const bool ell = d.geo_rows3 > 1;
  const int n3s = ell ? 1 : d.n3;
  const double* f = dbl + (b * Q + l) * size_t(d.ncell);
  double s = 0.0;
  for (int it = 0; it < d.nt; ++it)
    for (int k3 = 0; k3 < n3s; ++k3) s += f[(size_t(ir) * d.nt + it) * d.n3 + (ell ? i3 : k3)];
  const double mean = s / double(d.nt * n3s);
  float* rb = ref + b * Q * nrows;
  rb[ell ? l * nrows + row : row * Q + l] = float(mean);
}

cudaError_t launch_ref_from_state(const double* dbl, float* ref, const Dims& d, cudaStream_t s) {
  const size_t n = size_t(d.batch) * size_t(d.nr) * size_t(d.geo_rows3) * Q;
  k_ref_from_state<<<unsigned((n + 255) / 256), 256, 0, s>>>(dbl, ref, d);
  return cudaGetLastError();
}

cudaError_t launch_ref_table(int K, float* ref, const GeoDev<float>& geo, const double* sqrtg,
                             const double* base_uth, const double* rho_in, const double* u_in, const Dims& d,
                             int mode, cudaStream_t s) {
  const uint32_t n = uint32_t(d.batch) * uint32_t(d.nr) * uint32_t(d.geo_rows3);
  const uint32_t nb = (n + 255) / 256;
  switch (K) {
    case KFLAT: k_ref_table<KFLAT><<<nb, 256, 0, s>>>(ref, geo, sqrtg, base_uth, rho_in, u_in, d, mode); break;
    case KCYL: k_ref_table<KCYL><<<nb, 256, 0, s>>>(ref, geo, sqrtg, base_uth, rho_in, u_in, d, mode); break;
    case KELL: k_ref_table<KELL><<<nb, 256, 0, s>>>(ref, geo, sqrtg, base_uth, rho_in, u_in, d, mode); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <class S>
cudaError_t launch_stream_table_t(int K, float4* st, const float* ref, const InstParams<float>* inst,
                                  const void* fin, const Dims& d, cudaStream_t s) {
  const uint32_t n = uint32_t(d.batch) * uint32_t(d.nr) * uint32_t(d.st_rows3);
  const uint32_t nb = (n + 127) / 128;
  const S* f = static_cast<const S*>(fin);
  switch (K) {
    case KFLAT: k_stream_table<KFLAT, S><<<nb, 128, 0, s>>>(st, ref, inst, f, d); break;
    case KCYL: k_stream_table<KCYL, S><<<nb, 128, 0, s>>>(st, ref, inst, f, d); break;
    case KELL: k_stream_table<KELL, S><<<nb, 128, 0, s>>>(st, ref, inst, f, d); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_stream_table(int prec, int K, float4* st, const float* ref, const InstParams<float>* inst,
                                const void* fin, const Dims& d, cudaStream_t s) {
  if (!st || !ref || d.st != st) return cudaErrorInvalidValue;
  if (prec == 2) return launch_stream_table_t<__half>(K, st, ref, inst, fin, d, s);
  if (prec == 3) return launch_stream_table_t<__nv_bfloat16>(K, st, ref, inst, fin, d, s);
  return cudaErrorInvalidValue;
}

cudaError_t launch_diag(const double* rho, const double* u, double* rowmean, const double* geo64,
                        const Dims& d, double* partial, int nblk, double* out, cudaStream_t s) {
  const int rows = d.batch * d.nr * d.nt;
  k_rowmean<<<(rows + 255) / 256, 256, 0, s>>>(u, rowmean, d);
  k_diag_partial<<<dim3(nblk, d.batch), DIAG_THREADS, 0, s>>>(rho, u, rowmean, geo64, d, partial,
                                                              nblk);
  k_diag_final<<<d.batch, DIAG_THREADS, 0, s>>>(partial, nblk, out);
  return cudaGetLastError();
}

}  // namespace lbgm
