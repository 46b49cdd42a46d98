// Per-voxel kernels of Alg. 1 (Sec. III-C): the fused primal step (steps 2-7
// except the l1 thresholds), the fused dual step (steps 3-4 finish, 12, 13), the
// scalar finish of step 14 and the stop rule (eq. StopCri_simulated), and the
// layout helpers.  All are HBM-bound streams over [N1][N2][N3p] cubes.
#include <math.h>
#include "s3ttv_internal.cuh"

namespace s3ttv {
namespace {

// Block-wide sum of two doubles (blockDim.x a multiple of 32, <= 1024).
template <int NV>
__device__ void block_sum(double (&v)[NV], double (*red)[32]) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(kFull, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) red[k][w] = v[k];
  __syncthreads();
  if (w == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      v[k] = lane < nw ? red[k][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(kFull, v[k], o);
    }
  }
}

__device__ __forceinline__ void hist_add(unsigned *cnt, float *sum, float z) {
  const unsigned bits = __float_as_uint(z) & 0x7fffffffu;
  if (bits == 0u) return;  // zeros never enter the active set
  const unsigned key = bits >> 20;
  atomicAdd(&cnt[key], 1u);
  atomicAdd(&sum[key], __uint_as_float(bits));
}

// Alg. 1 steps 2-7 for u, and the arguments of the projections of steps 3-4.
//   u+   = P_[lo,hi](u - gu (D_s^T (D_v^T Zv + D_h^T Zh) + y3))     (step 2)
//   ubar = 2 u+ - u                                                  (step 5)
//   zs   = s - gs y3,   zt = t - gt (D_v^T y2 + y3)                 (steps 3, 4)
// with y3 = c3 d and Z = sum_l P_l^T Y_l.  Also: sum (u+ - u)^2 and sum u^2 for
// the stop rule, the first radix level of |zs| and |zt|, and zeroing of the next
// Z accumulator.
__global__ void __launch_bounds__(256) primal_kernel(PrimalArgs a) {
  __shared__ unsigned s_cnt[2 * kHistBins];
  __shared__ float s_sum[2 * kHistBins];
  __shared__ double s_red[2][32];
  if (a.sc->done) return;
  for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) {
    s_cnt[i] = 0u;
    s_sum[i] = 0.f;
  }
  __syncthreads();
  const Dims dm = a.dm;
  const long long N3p = dm.N3p;
  const float c3 = (float)a.sc->c3;
  float du2 = 0.f, u2 = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < dm.Np; idx += stride) {
    const long long pix = idx / N3p;
    const int b = (int)(idx - pix * N3p);
    a.Znv[idx] = 0.f;
    a.Znh[idx] = 0.f;
    if (b >= dm.N3) {
      a.ubar[idx] = 0.f;
      a.zs[idx] = 0.f;
      a.zt[idx] = 0.f;
      continue;
    }
    const int i = (int)(pix / dm.N2), j = (int)(pix - (long long)i * dm.N2);
    const long long pim = ((long long)(i == 0 ? dm.N1 - 1 : i - 1) * dm.N2 + j) * N3p;
    const long long pjm = ((long long)i * dm.N2 + (j == 0 ? dm.N2 - 1 : j - 1)) * N3p;
    const long long p0 = pix * N3p;
    const int bm = b == 0 ? dm.N3 - 1 : b - 1;
    const float w_b = (a.Zv[pim + b] - a.Zv[p0 + b]) + (a.Zh[pjm + b] - a.Zh[p0 + b]);
    const float w_bm = (a.Zv[pim + bm] - a.Zv[p0 + bm]) + (a.Zh[pjm + bm] - a.Zh[p0 + bm]);
    const float grad = w_bm - w_b;  // (D_s^T w)[b] = w[b-1] - w[b]
    const float y3 = c3 * a.d[idx];
    const float u = a.u[idx];
    const float x = u - a.gu * (grad + y3);
    const float un = (x != x) ? x : fminf(fmaxf(x, a.lo), a.hi);  // NaN stays visible
    a.u[idx] = un;
    a.ubar[idx] = 2.f * un - u;
    const float zs = a.s[idx] - a.gs * y3;
    const float zt = a.t[idx] - a.gt * ((a.y2[pim + b] - a.y2[idx]) + y3);
    a.zs[idx] = zs;
    a.zt[idx] = zt;
    const float dl = un - u;
    du2 = fmaf(dl, dl, du2);
    u2 = fmaf(u, u, u2);
    hist_add(s_cnt, s_sum, zs);
    hist_add(s_cnt + kHistBins, s_sum + kHistBins, zt);
  }
  double v[2] = {(double)du2, (double)u2};
  block_sum<2>(v, s_red);
  if (threadIdx.x == 0) {
    a.part[blockIdx.x] = v[0];
    a.part[gridDim.x + blockIdx.x] = v[1];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) {
    const unsigned c = s_cnt[i];
    if (c) {
      atomicAdd(&a.hcnt[i], c);
      atomicAdd(&a.hsum[i], (double)s_sum[i]);
    }
  }
}

// Steps 3-4 finish (soft thresholds found by the radix selection), steps 6-7,
// step 12 and step 13:
//   s+ = soft(zs, tau_s), t+ = soft(zt, tau_t), sbar = 2s+ - s, tbar = 2t+ - t,
//   y2 += g2 D_v tbar,   y3' = y3 + g3 (ubar + sbar + tbar),   d = y3'/g3 - v.
// Step 14 then sets y3 = g3 max(0, 1 - eps/||d||) d, i.e. only the scalar c3
// changes (finalize_kernel).  D_v tbar needs tbar of the pixel below, which is
// recomputed from zt and the old t there, so t is double-buffered.
__global__ void __launch_bounds__(256) dual_kernel(DualArgs a) {
  __shared__ double s_red[1][32];
  if (a.sc->done) return;
  const Dims dm = a.dm;
  const long long N3p = dm.N3p;
  const float c3 = (float)a.sc->c3;
  const float tau_s = a.sc->l1[0].tau, tau_t = a.sc->l1[1].tau;
  const float tls = a.sc->l1[0].tau_lo, tlt = a.sc->l1[1].tau_lo;
  const float inv_g3 = 1.f / a.g3;
  float d2 = 0.f;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < dm.Np; idx += stride) {
    const long long pix = idx / N3p;
    const int b = (int)(idx - pix * N3p);
    if (b >= dm.N3) {
      a.t_new[idx] = 0.f;
      continue;
    }
    const int i = (int)(pix / dm.N2), j = (int)(pix - (long long)i * dm.N2);
    const long long pip = ((long long)(i + 1 == dm.N1 ? 0 : i + 1) * dm.N2 + j) * N3p + b;
    const float sp = soft_threshold(a.zs[idx], tau_s, tls);
    const float sbar = 2.f * sp - a.s_old[idx];
    const float tp = soft_threshold(a.zt[idx], tau_t, tlt);
    const float tbar = 2.f * tp - a.t_old[idx];
    const float tbar_n = 2.f * soft_threshold(a.zt[pip], tau_t, tlt) - a.t_old[pip];
    a.y2[idx] = fmaf(a.g2, tbar_n - tbar, a.y2[idx]);
    const float y3p = fmaf(a.g3, a.ubar[idx] + sbar + tbar, c3 * a.d[idx]);
    const float dn = y3p * inv_g3 - a.v[idx];
    a.s_new[idx] = sp;
    a.t_new[idx] = tp;
    a.d[idx] = dn;
    d2 = fmaf(dn, dn, d2);
  }
  double v[1] = {(double)d2};
  block_sum<1>(v, s_red);
  if (threadIdx.x == 0) a.part[blockIdx.x] = v[0];
}

// Step 14's scalar (eq. prox_l2ball_constraint through Moreau) and the stop rule.
__global__ void __launch_bounds__(256) finalize_kernel(FinalizeArgs a) {
  __shared__ double s_red[3][32];
  Scalars *sc = a.sc;
  if (sc->done) return;
  double v[3] = {0.0, 0.0, 0.0};
  for (int i = threadIdx.x; i < a.grid_p; i += blockDim.x) {
    v[0] += a.part_primal[i];
    v[1] += a.part_primal[a.grid_p + i];
  }
  for (int i = threadIdx.x; i < a.grid_d; i += blockDim.x) v[2] += a.part_dual[i];
  block_sum<3>(v, s_red);
  if (threadIdx.x == 0) {
    const double du2 = v[0], u2 = v[1], d2 = v[2];
    const double nd = sqrt(d2);
    sc->c3 = nd > a.eps ? a.g3 * (1.0 - a.eps / nd) : 0.0;
    const double rel = u2 > 0.0 ? sqrt(du2) / sqrt(u2) : sqrt(du2);
    sc->rel = rel;
    sc->iter += 1;
    if (!isfinite(rel) || !isfinite(d2)) {
      sc->status = -4;
      sc->done = 1;
    } else if (rel < (double)sc->tol) {
      sc->status = 1;
      sc->done = 1;
    } else if (sc->iter >= sc->iter_limit) {
      sc->status = 2;
      sc->done = 1;
    }
  }
}

__global__ void pad_cube_kernel(const float *__restrict__ src, float *__restrict__ dst, Dims dm, float scale) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < dm.Np; idx += stride) {
    const long long pix = idx / dm.N3p;
    const int b = (int)(idx - pix * dm.N3p);
    dst[idx] = b < dm.N3 ? scale * src[pix * dm.N3 + b] : 0.f;
  }
}

__global__ void unpad_cube_kernel(const float *__restrict__ src, float *__restrict__ dst, Dims dm,
                                  const double *scale_dev) {
  const float scale = scale_dev ? (float)*scale_dev : 1.f;
  const long long n = dm.P * dm.N3;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < n; idx += stride) {
    const long long pix = idx / dm.N3;
    const int b = (int)(idx - pix * dm.N3);
    dst[idx] = scale * src[pix * dm.N3p + b];
  }
}

// External Y [L][n][2*N3] (column 2b + o) <-> internal [L][n][2][N3p].
__global__ void Y_to_internal_kernel(const float *__restrict__ ext, float *__restrict__ in, Dims dm, int n) {
  const long long total = dm.P * n * 2 * dm.N3p;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const long long row = idx / (2 * dm.N3p);
    const int rem = (int)(idx - row * 2 * dm.N3p);
    const int o = rem >= dm.N3p;
    const int b = rem - o * dm.N3p;
    in[idx] = b < dm.N3 ? ext[row * 2 * dm.N3 + 2 * b + o] : 0.f;
  }
}

__global__ void Y_to_external_kernel(const float *__restrict__ in, float *__restrict__ ext, Dims dm, int n) {
  const long long total = dm.P * n * 2 * dm.N3;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const long long row = idx / (2 * dm.N3);
    const int col = (int)(idx - row * 2 * dm.N3);
    const int b = col >> 1, o = col & 1;
    ext[idx] = in[row * 2 * dm.N3p + (long long)o * dm.N3p + b];
  }
}

// Z = sum_l P_l^T Y_l by gathering, for each pixel, the rows of the k^2 blocks
// that cover it (used when a caller replaces Y).
__global__ void Z_from_Y_kernel(const float *__restrict__ Y, float *__restrict__ Zv, float *__restrict__ Zh,
                                Dims dm, int k) {
  const int n = k * k;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < dm.Np; idx += stride) {
    const long long pix = idx / dm.N3p;
    const int b = (int)(idx - pix * dm.N3p);
    const int i = (int)(pix / dm.N2), j = (int)(pix - (long long)i * dm.N2);
    float zv = 0.f, zh = 0.f;
    for (int aa = 0; aa < k; ++aa) {
      const int ii = (i - aa + dm.N1) % dm.N1;
      for (int cc = 0; cc < k; ++cc) {
        const int jj = (j - cc + dm.N2) % dm.N2;
        const long long base = (((long long)ii * dm.N2 + jj) * n + aa * k + cc) * 2 * dm.N3p;
        zv += Y[base + b];
        zh += Y[base + dm.N3p + b];
      }
    }
    Zv[idx] = zv;
    Zh[idx] = zh;
  }
}

// Fv = D_v D_s ubar and Fh = D_h D_s ubar: the second-order differences the
// structure tensors of eq. (SSST) are cut from, formed once per pass.
__global__ void xfield_kernel(const float *__restrict__ ubar, float *__restrict__ Fv, float *__restrict__ Fh,
                              Dims dm) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < dm.Np; idx += stride) {
    const long long pix = idx / dm.N3p;
    const int b = (int)(idx - pix * dm.N3p);
    if (b >= dm.N3) {
      Fv[idx] = 0.f;
      Fh[idx] = 0.f;
      continue;
    }
    const int i = (int)(pix / dm.N2), j = (int)(pix - (long long)i * dm.N2);
    const int bn = b + 1 == dm.N3 ? 0 : b + 1;
    const long long p0 = pix * dm.N3p;
    const long long pv = ((long long)(i + 1 == dm.N1 ? 0 : i + 1) * dm.N2 + j) * dm.N3p;
    const long long ph = ((long long)i * dm.N2 + (j + 1 == dm.N2 ? 0 : j + 1)) * dm.N3p;
    const float ds0 = ubar[p0 + bn] - ubar[p0 + b];
    Fv[idx] = (ubar[pv + bn] - ubar[pv + b]) - ds0;
    Fh[idx] = (ubar[ph + bn] - ubar[ph + b]) - ds0;
  }
}

__global__ void init_scalars_kernel(Scalars *sc, double alpha, double beta) {
  Scalars s = {};
  s.l1[0].radius = alpha;
  s.l1[1].radius = beta;
  *sc = s;
}

int grid_for(long long n) {
  long long g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  return (int)g;
}

}  // namespace

cudaError_t launch_primal(const PrimalArgs &a, int grid, cudaStream_t st) {
  primal_kernel<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dual(const DualArgs &a, int grid, cudaStream_t st) {
  dual_kernel<<<grid, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t st) {
  finalize_kernel<<<1, 256, 0, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_pad_cube(const float *src, float *dst, Dims dm, float scale, cudaStream_t st) {
  pad_cube_kernel<<<grid_for(dm.Np), 256, 0, st>>>(src, dst, dm, scale);
  return cudaGetLastError();
}

cudaError_t launch_unpad_cube(const float *src, float *dst, Dims dm, const double *scale_dev, cudaStream_t st) {
  unpad_cube_kernel<<<grid_for(dm.P * dm.N3), 256, 0, st>>>(src, dst, dm, scale_dev);
  return cudaGetLastError();
}

cudaError_t launch_Y_to_internal(const float *ext, float *in, Dims dm, int k, cudaStream_t st) {
  Y_to_internal_kernel<<<grid_for(dm.P * k * k * 2 * dm.N3p), 256, 0, st>>>(ext, in, dm, k * k);
  return cudaGetLastError();
}

cudaError_t launch_Y_to_external(const float *in, float *ext, Dims dm, int k, cudaStream_t st) {
  Y_to_external_kernel<<<grid_for(dm.P * k * k * 2 * dm.N3), 256, 0, st>>>(in, ext, dm, k * k);
  return cudaGetLastError();
}

cudaError_t launch_xfield(const float *ubar, float *Fv, float *Fh, Dims dm, int grid, cudaStream_t st) {
  xfield_kernel<<<grid, 256, 0, st>>>(ubar, Fv, Fh, dm);
  return cudaGetLastError();
}

cudaError_t launch_Z_from_Y(const float *Y, float *Zv, float *Zh, Dims dm, int k, cudaStream_t st) {
  Z_from_Y_kernel<<<grid_for(dm.Np), 256, 0, st>>>(Y, Zv, Zh, dm, k);
  return cudaGetLastError();
}

cudaError_t launch_init_scalars(Scalars *sc, double alpha, double beta, cudaStream_t st) {
  init_scalars_kernel<<<1, 1, 0, st>>>(sc, alpha, beta);
  return cudaGetLastError();
}

}  // namespace s3ttv
