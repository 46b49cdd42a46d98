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

// Work unit of primal_kernel and dual_kernel: one float4 chunk (4 consecutive
// bands) of one pixel; chunk c is pixel c / C4, bands 4 (c mod C4) .. + 3.
// The host admits cubes of fewer than 2^31 chunks, so the index arithmetic is
// 32-bit.
__device__ __forceinline__ float4 ld4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void st4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float comp(const float4 &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }

// Alg. 1 steps 2-7 for u, and the arguments of the projections of steps 3-4.
//   u+   = P_[lo,hi](u - gu (D_s^T (D_v^T Zv + D_h^T Zh) + y3))     (step 2)
//   ubar = 2 u+ - u                                                  (step 5)
//   zs   = s - gs y3,   zt = t - gt (D_v^T y2 + y3)                 (steps 3, 4)
// with y3 = c3 d and Z = sum_l P_l^T Y_l.  Also: sum (u+ - u)^2 and sum u^2 for
// the stop rule, the first radix level of |zs| and |zt|, and zeroing of the next
// Z accumulator.  EXTRA: 0 S3TTV, STV, SSTV; 1 HSSTV (+ omega D^T of the
// first-order dual pair); 2 SSST (+ D_s^T Zs, and Zns zeroed).
template <int EXTRA>
__global__ void __launch_bounds__(256) primal_kernel(PrimalArgs a) {
  __shared__ unsigned s_cnt[2 * kHistBins];
  __shared__ float s_sum[2 * kHistBins];
  __shared__ double s_red[2][32];
  if (a.sc->done) return;
  // this pass's FP64 re-solve queue starts empty (the block dual runs after this
  // kernel, the previous pass's re-solve before it)
  if (blockIdx.x == 0 && threadIdx.x == 0) a.sc->fb_count = 0u;
  for (int i = threadIdx.x; i < 2 * kHistBins; i += blockDim.x) {
    s_cnt[i] = 0u;
    s_sum[i] = 0.f;
  }
  __syncthreads();
  const Dims dm = a.dm;
  const int N3p = dm.N3p, C4 = N3p >> 2, N2 = dm.N2;
  const int nch = (int)(dm.P * C4);
  const float c3 = (float)a.sc->c3;
  float du2 = 0.f, u2 = 0.f;
  const float4 zero4 = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nch; c += gridDim.x * blockDim.x) {
    const int pix = (unsigned)c / (unsigned)C4, q = c - pix * C4, b0 = q << 2;
    const int i = (unsigned)pix / (unsigned)N2, j = pix - i * N2;
    const size_t p0 = (size_t)pix * N3p + b0;
    const size_t pim = ((size_t)(i == 0 ? dm.N1 - 1 : i - 1) * N2 + j) * N3p + b0;
    const size_t pjm = ((size_t)i * N2 + (j == 0 ? N2 - 1 : j - 1)) * N3p + b0;
    st4(a.Znv + p0, zero4);
    st4(a.Znh + p0, zero4);
    if (EXTRA == 2) st4(a.Zns + p0, zero4);
    // w = D_v^T Zv + D_h^T Zh at bands b0..b0+3 and at the band before b0
    // (periodic over the N3 true bands)
    const float4 zv = ld4(a.Zv + p0), zvm = ld4(a.Zv + pim), zh = ld4(a.Zh + p0), zhm = ld4(a.Zh + pjm);
    const float w[4] = {(zvm.x - zv.x) + (zhm.x - zh.x), (zvm.y - zv.y) + (zhm.y - zh.y),
                        (zvm.z - zv.z) + (zhm.z - zh.z), (zvm.w - zv.w) + (zhm.w - zh.w)};
    const long long o = (b0 == 0 ? dm.N3 - 1 : b0 - 1) - b0;  // to the band before (periodic)
    const float wbm = (a.Zv[(long long)pim + o] - a.Zv[(long long)p0 + o]) +
                      (a.Zh[(long long)pjm + o] - a.Zh[(long long)p0 + o]);
    float4 zs4 = zero4;
    float zsm = 0.f;
    if (EXTRA == 2) {  // SSST's third dual part at bands b0..b0+3 and the band before
      zs4 = ld4(a.Zs + p0);
      zsm = a.Zs[(long long)p0 + o];
    }
    const float4 d4 = ld4(a.d + p0), u4 = ld4(a.u + p0), s4 = ld4(a.s + p0), t4 = ld4(a.t + p0);
    const float4 y2c = ld4(a.y2 + p0), y2m = ld4(a.y2 + pim);
    float un[4], ub[4], zs[4], zt[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (b0 + e < dm.N3) {
        // (D_s^T w)[b] = w[b-1] - w[b]; STV's first-order term has no D_s
        float grad = a.no_ds ? w[e] : (e == 0 ? wbm : w[e - 1]) - w[e];
        if (EXTRA == 1)  // HSSTV: + omega D^T (Y1v, Y1h), first-order, no D_s
          grad = fmaf(a.w1, (a.Z1v[pim + e] - a.Z1v[p0 + e]) + (a.Z1h[pjm + e] - a.Z1h[p0 + e]), grad);
        if (EXTRA == 2)  // SSST: + D_s^T Zs, (D_s^T z)[b] = z[b-1] - z[b] (periodic)
          grad += (e == 0 ? zsm : comp(zs4, e - 1)) - comp(zs4, e);
        const float y3 = c3 * comp(d4, e);
        const float u = comp(u4, e);
        const float x = u - a.gu * (grad + y3);
        const float v = (x != x) ? x : fminf(fmaxf(x, a.lo), a.hi);  // NaN stays visible
        un[e] = v;
        ub[e] = 2.f * v - u;
        zs[e] = comp(s4, e) - a.gs * y3;
        zt[e] = comp(t4, e) - a.gt * ((comp(y2m, e) - comp(y2c, e)) + y3);
        const float dl = v - u;
        du2 = fmaf(dl, dl, du2);
        u2 = fmaf(u, u, u2);
        hist_add(s_cnt, s_sum, zs[e]);
        hist_add(s_cnt + kHistBins, s_sum + kHistBins, zt[e]);
      } else {  // padding bands stay 0
        un[e] = comp(u4, e);
        ub[e] = zs[e] = zt[e] = 0.f;
      }
    }
    st4(a.u + p0, make_float4(un[0], un[1], un[2], un[3]));
    st4(a.ubar + p0, make_float4(ub[0], ub[1], ub[2], ub[3]));
    st4(a.zs + p0, make_float4(zs[0], zs[1], zs[2], zs[3]));
    st4(a.zt + p0, make_float4(zt[0], zt[1], zt[2], zt[3]));
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

// Alg. 1 steps 3-4 finish (soft thresholds), 6-7, 12 and 13:
//   s+ = S_tau_s(zs), t+ = S_tau_t(zt), sbar = 2 s+ - s, tbar = 2 t+ - t
//   y2 += g2 D_v tbar                                                (step 12)
//   y3' = y3 + g3 (ubar + sbar + tbar),  d = y3' / g3 - v            (step 13)
// (step 14 scales d by the scalar c3 of finalize_kernel), and sum d^2.
__global__ void __launch_bounds__(256) dual_kernel(DualArgs a) {
  __shared__ double s_red[1][32];
  if (a.sc->done) return;
  const Dims dm = a.dm;
  const int N3p = dm.N3p, C4 = N3p >> 2, N2 = dm.N2;
  const int nch = (int)(dm.P * C4);
  const float c3 = (float)a.sc->c3;
  const float tau_s = a.sc->l1[0].tau, tau_t = a.sc->l1[1].tau;
  const float tls = a.sc->l1[0].tau_lo, tlt = a.sc->l1[1].tau_lo;
  const float inv_g3 = 1.f / a.g3;
  float d2 = 0.f;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nch; c += gridDim.x * blockDim.x) {
    const int pix = (unsigned)c / (unsigned)C4, q = c - pix * C4, b0 = q << 2;
    const int i = (unsigned)pix / (unsigned)N2, j = pix - i * N2;
    const size_t p0 = (size_t)pix * N3p + b0;
    const size_t pip = ((size_t)(i + 1 == dm.N1 ? 0 : i + 1) * N2 + j) * N3p + b0;
    const float4 zs4 = ld4(a.zs + p0), zt4 = ld4(a.zt + p0), ztn = ld4(a.zt + pip);
    const float4 so4 = ld4(a.s_old + p0), to4 = ld4(a.t_old + p0), ton = ld4(a.t_old + pip);
    const float4 y24 = ld4(a.y2 + p0), ub4 = ld4(a.ubar + p0), d4 = ld4(a.d + p0), v4 = ld4(a.v + p0);
    float sp[4], tp[4], y2n[4], dn[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (b0 + e < dm.N3) {
        sp[e] = soft_threshold(comp(zs4, e), tau_s, tls);
        const float sbar = 2.f * sp[e] - comp(so4, e);
        tp[e] = soft_threshold(comp(zt4, e), tau_t, tlt);
        const float tbar = 2.f * tp[e] - comp(to4, e);
        const float tbar_n = 2.f * soft_threshold(comp(ztn, e), tau_t, tlt) - comp(ton, e);
        y2n[e] = fmaf(a.g2, tbar_n - tbar, comp(y24, e));
        const float y3p = fmaf(a.g3, comp(ub4, e) + sbar + tbar, c3 * comp(d4, e));
        dn[e] = y3p * inv_g3 - comp(v4, e);
        d2 = fmaf(dn[e], dn[e], d2);
      } else {  // padding bands stay 0
        sp[e] = tp[e] = 0.f;
        y2n[e] = comp(y24, e);
        dn[e] = comp(d4, e);
      }
    }
    st4(a.s_new + p0, make_float4(sp[0], sp[1], sp[2], sp[3]));
    st4(a.t_new + p0, make_float4(tp[0], tp[1], tp[2], tp[3]));
    st4(a.y2 + p0, make_float4(y2n[0], y2n[1], y2n[2], y2n[3]));
    st4(a.d + p0, make_float4(dn[0], dn[1], dn[2], dn[3]));
  }
  double v[1] = {(double)d2};
  block_sum<1>(v, s_red);
  if (threadIdx.x == 0) a.part[blockIdx.x] = v[0];
}

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
// External block duals: paper layout [L][k^2][2 N3] with interleaved columns
// (v_b, h_b); stacked layout [L][2 k^2][N3] (row 2r + o, band b).  Internal:
// [L][k^2][2][N3p] for both.
__global__ void Y_to_internal_kernel(const float *__restrict__ ext, float *__restrict__ in, Dims dm, int n,
                                     int stacked, int parts) {
  const long long total = dm.P * n * parts * dm.N3p;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const long long row = idx / (parts * dm.N3p);
    const int rem = (int)(idx - row * parts * dm.N3p);
    const int o = rem / dm.N3p;
    const int b = rem - o * dm.N3p;
    in[idx] = b < dm.N3 ? ext[stacked ? (2 * row + o) * dm.N3 + b : row * parts * dm.N3 + parts * b + o] : 0.f;
  }
}

__global__ void Y_to_external_kernel(const float *__restrict__ in, float *__restrict__ ext, Dims dm, int n,
                                     int stacked, int parts) {
  const long long total = dm.P * n * parts * dm.N3;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
    const long long row = idx / (parts * dm.N3);
    const int col = (int)(idx - row * parts * dm.N3);
    const int b = stacked ? col % dm.N3 : col / parts, o = stacked ? col / dm.N3 : col % parts;
    ext[idx] = in[row * parts * dm.N3p + (long long)o * dm.N3p + b];
  }
}

// Z = sum_l P_l^T Y_l by gathering, for each pixel, the rows of the k^2 blocks
// that cover it (used when a caller replaces Y).
__global__ void Z_from_Y_kernel(const float *__restrict__ Y, float *__restrict__ Zv, float *__restrict__ Zh,
                                Dims dm, int k, float *__restrict__ Zs) {
  const int parts = Zs ? 3 : 2;
  const int n = k * k;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < dm.Np; idx += stride) {
    const long long pix = idx / dm.N3p;
    const int b = (int)(idx - pix * dm.N3p);
    const int i = (int)(pix / dm.N2), j = (int)(pix - (long long)i * dm.N2);
    float zv = 0.f, zh = 0.f, zs = 0.f;
    for (int aa = 0; aa < k; ++aa) {
      const int ii = (i - aa + dm.N1) % dm.N1;
      for (int cc = 0; cc < k; ++cc) {
        const int jj = (j - cc + dm.N2) % dm.N2;
        const long long base = (((long long)ii * dm.N2 + jj) * n + aa * k + cc) * parts * dm.N3p;
        zv += Y[base + b];
        zh += Y[base + dm.N3p + b];
        if (Zs) zs += Y[base + 2 * dm.N3p + b];
      }
    }
    Zv[idx] = zv;
    Zh[idx] = zh;
    if (Zs) Zs[idx] = zs;
  }
}

// Fv = D_v D_s ubar and Fh = D_h D_s ubar: the second-order differences the
// structure tensors of eq. (SSST) are cut from, formed once per pass.
__global__ void xfield_kernel(const float *__restrict__ ubar, float *__restrict__ Fv, float *__restrict__ Fh,
                              Dims dm, int open_s, int first_order, float *__restrict__ Fs) {
  const int N3p = dm.N3p, C4 = N3p >> 2, N2 = dm.N2;
  const int nch = (int)(dm.P * C4);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nch; c += gridDim.x * blockDim.x) {
    const int pix = (unsigned)c / (unsigned)C4, q = c - pix * C4, b0 = q << 2;
    const int i = (unsigned)pix / (unsigned)N2, j = pix - i * N2;
    const size_t p0 = (size_t)pix * N3p;
    const size_t pv = ((size_t)(i + 1 == dm.N1 ? 0 : i + 1) * N2 + j) * N3p;
    const size_t ph = ((size_t)i * N2 + (j + 1 == N2 ? 0 : j + 1)) * N3p;
    // bands b0..b0+3 and the band after the chunk (periodic over the N3 true bands)
    const float4 x0 = ld4(ubar + p0 + b0), xv = ld4(ubar + pv + b0), xh = ld4(ubar + ph + b0);
    const int nb = b0 + 4 < dm.N3 ? b0 + 4 : 0;
    const float n0 = ubar[p0 + nb], nv = ubar[pv + nb], nh = ubar[ph + nb];
    float fv[4], fh[4], fs[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      fs[e] = 0.f;
      if (b0 + e < dm.N3 - open_s) {  // open D_s: no difference past the last band
        const bool in = e < 3 && b0 + e + 1 < dm.N3;
        if (first_order) {  // STV: D_v u, D_h u (SSST: and D_s u)
          fv[e] = comp(xv, e) - comp(x0, e);
          fh[e] = comp(xh, e) - comp(x0, e);
          fs[e] = (in ? comp(x0, e + 1) : n0) - comp(x0, e);
        } else {
          const float ds0 = (in ? comp(x0, e + 1) : n0) - comp(x0, e);
          fv[e] = ((in ? comp(xv, e + 1) : nv) - comp(xv, e)) - ds0;
          fh[e] = ((in ? comp(xh, e + 1) : nh) - comp(xh, e)) - ds0;
        }
      } else {
        fv[e] = fh[e] = 0.f;
      }
    }
    st4(Fv + p0 + b0, make_float4(fv[0], fv[1], fv[2], fv[3]));
    st4(Fh + p0 + b0, make_float4(fh[0], fh[1], fh[2], fh[3]));
    if (Fs) st4(Fs + p0 + b0, make_float4(fs[0], fs[1], fs[2], fs[3]));
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
  if (a.Zs) primal_kernel<2><<<grid, 256, 0, st>>>(a);
  else if (a.Z1v) primal_kernel<1><<<grid, 256, 0, st>>>(a);
  else primal_kernel<0><<<grid, 256, 0, st>>>(a);
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

// SSTV's dual step (the l1 norm of D D_s u in place of the block nuclear
// norms): Y' = Y + gamma_Y (D_v D_s ubar, D_h D_s ubar), and the conjugate prox
// of the l1 norm (eq. ProxConjugate) is the projection onto the unit l_inf
// ball, Y = clip(Y', -1, 1).  Y = (Yv, Yh) are internal cubes, and
// Z = sum_l P_l^T Y_l becomes Y itself: written to (Zv, Zh).
__global__ void sstv_dual_kernel(const float *__restrict__ ubar, float *__restrict__ Yv, float *__restrict__ Yh,
                                 float *__restrict__ Zv, float *__restrict__ Zh, Dims dm, float gY) {
  const int N3p = dm.N3p, C4 = N3p >> 2, N2 = dm.N2;
  const int nch = (int)(dm.P * C4);
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nch; c += gridDim.x * blockDim.x) {
    const int pix = (unsigned)c / (unsigned)C4, q = c - pix * C4, b0 = q << 2;
    const int i = (unsigned)pix / (unsigned)N2, j = pix - i * N2;
    const size_t p0 = (size_t)pix * N3p;
    const size_t pv = ((size_t)(i + 1 == dm.N1 ? 0 : i + 1) * N2 + j) * N3p;
    const size_t ph = ((size_t)i * N2 + (j + 1 == N2 ? 0 : j + 1)) * N3p;
    const float4 x0 = ld4(ubar + p0 + b0), xv = ld4(ubar + pv + b0), xh = ld4(ubar + ph + b0);
    const int nb = b0 + 4 < dm.N3 ? b0 + 4 : 0;
    const float n0 = ubar[p0 + nb], nv = ubar[pv + nb], nh = ubar[ph + nb];
    const float4 yv4 = ld4(Yv + p0 + b0), yh4 = ld4(Yh + p0 + b0);
    float yv[4], yh[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (b0 + e < dm.N3) {
        const bool in = e < 3 && b0 + e + 1 < dm.N3;
        const float ds0 = (in ? comp(x0, e + 1) : n0) - comp(x0, e);
        const float fv = ((in ? comp(xv, e + 1) : nv) - comp(xv, e)) - ds0;
        const float fh = ((in ? comp(xh, e + 1) : nh) - comp(xh, e)) - ds0;
        yv[e] = fminf(fmaxf(fmaf(gY, fv, comp(yv4, e)), -1.f), 1.f);
        yh[e] = fminf(fmaxf(fmaf(gY, fh, comp(yh4, e)), -1.f), 1.f);
      } else {
        yv[e] = yh[e] = 0.f;
      }
    }
    const float4 ov = make_float4(yv[0], yv[1], yv[2], yv[3]), oh = make_float4(yh[0], yh[1], yh[2], yh[3]);
    st4(Yv + p0 + b0, ov);
    st4(Yh + p0 + b0, oh);
    st4(Zv + p0 + b0, ov);
    st4(Zh + p0 + b0, oh);
  }
}

// HSSTV's dual step: the four parts (D_v D_s ubar, D_h D_s ubar, omega D_v ubar,
// omega D_h ubar) added to Y with gamma_Y, then the conjugate prox of the l1
// norm (l12 = 0: clip every entry to [-1, 1]) or of the l1,2 norm over each
// voxel's four entries (l12 = 1: scale the 4-vector into the unit l2 ball).
// Y holds four internal cubes; the second-order pair is also written to Z.
__global__ void hsstv_dual_kernel(const float *__restrict__ ubar, float *__restrict__ Y, float *__restrict__ Zv,
                                  float *__restrict__ Zh, Dims dm, float gY, float omega, int l12) {
  const int N3p = dm.N3p, C4 = N3p >> 2, N2 = dm.N2;
  const int nch = (int)(dm.P * C4);
  const size_t Np = (size_t)dm.Np;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nch; c += gridDim.x * blockDim.x) {
    const int pix = (unsigned)c / (unsigned)C4, q = c - pix * C4, b0 = q << 2;
    const int i = (unsigned)pix / (unsigned)N2, j = pix - i * N2;
    const size_t p0 = (size_t)pix * N3p;
    const size_t pv = ((size_t)(i + 1 == dm.N1 ? 0 : i + 1) * N2 + j) * N3p;
    const size_t ph = ((size_t)i * N2 + (j + 1 == N2 ? 0 : j + 1)) * N3p;
    const float4 x0 = ld4(ubar + p0 + b0), xv = ld4(ubar + pv + b0), xh = ld4(ubar + ph + b0);
    const int nb = b0 + 4 < dm.N3 ? b0 + 4 : 0;
    const float n0 = ubar[p0 + nb], nv = ubar[pv + nb], nh = ubar[ph + nb];
    float4 y4[4];
#pragma unroll
    for (int m = 0; m < 4; ++m) y4[m] = ld4(Y + m * Np + p0 + b0);
    float o[4][4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      if (b0 + e < dm.N3) {
        const bool in = e < 3 && b0 + e + 1 < dm.N3;
        const float ds0 = (in ? comp(x0, e + 1) : n0) - comp(x0, e);
        const float f[4] = {((in ? comp(xv, e + 1) : nv) - comp(xv, e)) - ds0,
                            ((in ? comp(xh, e + 1) : nh) - comp(xh, e)) - ds0,
                            omega * (comp(xv, e) - comp(x0, e)), omega * (comp(xh, e) - comp(x0, e))};
        float yp[4], s2 = 0.f;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          yp[m] = fmaf(gY, f[m], comp(y4[m], e));
          s2 = fmaf(yp[m], yp[m], s2);
        }
        const float sc = l12 && s2 > 1.f ? rsqrtf(s2) : 1.f;
#pragma unroll
        for (int m = 0; m < 4; ++m) o[m][e] = l12 ? yp[m] * sc : fminf(fmaxf(yp[m], -1.f), 1.f);
      } else {
#pragma unroll
        for (int m = 0; m < 4; ++m) o[m][e] = 0.f;
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) st4(Y + m * Np + p0 + b0, make_float4(o[m][0], o[m][1], o[m][2], o[m][3]));
    st4(Zv + p0 + b0, make_float4(o[0][0], o[0][1], o[0][2], o[0][3]));
    st4(Zh + p0 + b0, make_float4(o[1][0], o[1][1], o[1][2], o[1][3]));
  }
}

cudaError_t launch_hsstv_dual(const float *ubar, float *Y, float *Zv, float *Zh, Dims dm, float gY, float omega,
                              int l12, int grid, cudaStream_t st) {
  hsstv_dual_kernel<<<grid, 256, 0, st>>>(ubar, Y, Zv, Zh, dm, gY, omega, l12);
  return cudaGetLastError();
}

cudaError_t launch_sstv_dual(const float *ubar, float *Yv, float *Yh, float *Zv, float *Zh, Dims dm, float gY,
                             int grid, cudaStream_t st) {
  sstv_dual_kernel<<<grid, 256, 0, st>>>(ubar, Yv, Yh, Zv, Zh, dm, gY);
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

cudaError_t launch_Y_to_internal(const float *ext, float *in, Dims dm, int k, cudaStream_t st, int stacked,
                                 int parts) {
  Y_to_internal_kernel<<<grid_for(dm.P * k * k * parts * dm.N3p), 256, 0, st>>>(ext, in, dm, k * k, stacked, parts);
  return cudaGetLastError();
}

cudaError_t launch_Y_to_external(const float *in, float *ext, Dims dm, int k, cudaStream_t st, int stacked,
                                 int parts) {
  Y_to_external_kernel<<<grid_for(dm.P * k * k * parts * dm.N3), 256, 0, st>>>(in, ext, dm, k * k, stacked, parts);
  return cudaGetLastError();
}

cudaError_t launch_xfield(const float *ubar, float *Fv, float *Fh, Dims dm, int grid, cudaStream_t st, int open_s,
                          int first_order, float *Fs) {
  xfield_kernel<<<grid, 256, 0, st>>>(ubar, Fv, Fh, dm, open_s, first_order, Fs);
  return cudaGetLastError();
}

cudaError_t launch_Z_from_Y(const float *Y, float *Zv, float *Zh, Dims dm, int k, cudaStream_t st, float *Zs) {
  Z_from_Y_kernel<<<grid_for(dm.Np), 256, 0, st>>>(Y, Zv, Zh, dm, k, Zs);
  return cudaGetLastError();
}

cudaError_t launch_init_scalars(Scalars *sc, double alpha, double beta, cudaStream_t st) {
  init_scalars_kernel<<<1, 1, 0, st>>>(sc, alpha, beta);
  return cudaGetLastError();
}

}  // namespace s3ttv
