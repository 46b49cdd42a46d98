// Projection onto the l1 ball {x : ||x||_1 <= r} (Alg. 1 steps 3-4; the paper
// cites Condat's fast l1-ball projection and gives it O(N log N) in Table II).
//
// The projection is sign(x) max(|x| - tau, 0) with the unique tau >= 0 solving
// h(tau) = sum_i max(|x_i| - tau, 0) = r (tau = 0 when ||x||_1 <= r).  Instead of
// sorting, the threshold is found by radix selection over the 31 magnitude bits
// of the FP32 values, which orders them exactly like their values: three
// histogram passes (11, 11 and 9 bits) each keep the bin whose lower edge is the
// last one with h >= r.  After the third level every bin holds a single value,
// the active set {|x| > tau} is exactly the elements above the chosen bin, and
// tau = (sum of the active |x| - r) / (their count), evaluated in FP64.
#include <math.h>
#include "s3ttv_internal.cuh"

namespace s3ttv {
namespace {

__global__ void __launch_bounds__(256) l1_hist_kernel(L1Args a, int level) {
  __shared__ unsigned s_cnt[kHistBins];
  __shared__ float s_sum[kHistBins];
  const int pb = blockIdx.y;
  if (a.sc->done) return;
  const L1State st = a.sc->l1[pb];
  if (level > 1 && st.mode != 0) return;
  const int bits = l1_level_bits(level), shift = l1_level_shift(level);
  const int nb = 1 << bits;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    s_cnt[i] = 0u;
    s_sum[i] = 0.f;
  }
  __syncthreads();
  const unsigned mask = (unsigned)nb - 1u;
  const unsigned prefix = level == 1 ? 0u : st.prefix;
  const int pshift = bits + shift;
  const float *x = a.x[pb];
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < a.n; idx += stride) {
    const unsigned ub = __float_as_uint(x[idx]) & 0x7fffffffu;
    if (ub == 0u) continue;
    if ((ub >> pshift) != prefix) continue;
    const unsigned key = (ub >> shift) & mask;
    atomicAdd(&s_cnt[key], 1u);
    atomicAdd(&s_sum[key], __uint_as_float(ub));
  }
  __syncthreads();
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    const unsigned c = s_cnt[i];
    if (c) {
      atomicAdd(&a.hcnt[pb * kHistBins + i], c);
      atomicAdd(&a.hsum[pb * kHistBins + i], (double)s_sum[i]);
    }
  }
}

// One CTA per problem: narrow the threshold by one radix level and clear the
// histogram for its next use.
__global__ void __launch_bounds__(1024) l1_scan_kernel(L1Args a, int level) {
  __shared__ unsigned long long s_wc[32];
  __shared__ double s_ws[32];
  __shared__ int s_best;
  __shared__ unsigned long long s_cx;
  __shared__ double s_sx;
  __shared__ L1State s_st;
  const int pb = blockIdx.x;
  if (a.sc->done) return;
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  unsigned *cnt = a.hcnt + pb * kHistBins;
  double *sum = a.hsum + pb * kHistBins;
  const int bits = l1_level_bits(level), shift = l1_level_shift(level);
  const int nb = 1 << bits;
  if (tid == 0) {
    L1State st = a.sc->l1[pb];
    if (level == 1) {
      st.S_above = 0.0;
      st.C_above = 0ull;
      st.prefix = 0u;
      st.mode = 0;
      st.tau = 0.f;
      st.tau_lo = 0.f;
    }
    s_st = st;
    s_best = -1;
  }
  __syncthreads();
  // Thread tid owns bins nb-1-2tid and nb-2-2tid (counted from the top).
  unsigned long long c[2] = {0ull, 0ull};
  double sm[2] = {0.0, 0.0};
  int bin[2] = {nb - 1 - 2 * tid, nb - 2 - 2 * tid};
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    if (bin[e] >= 0) {
      c[e] = cnt[bin[e]];
      sm[e] = sum[bin[e]];
      cnt[bin[e]] = 0u;
      sum[bin[e]] = 0.0;
    }
  }
  if (s_st.mode != 0) return;  // decided at an earlier level (uniform)
  // Inclusive scan from the top: suffix sums over bins >= bin[e].
  unsigned long long ci = c[0] + c[1];
  double si = sm[0] + sm[1];
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long cu = __shfl_up_sync(kFull, ci, o);
    const double su = __shfl_up_sync(kFull, si, o);
    if (lane >= o) {
      ci += cu;
      si += su;
    }
  }
  if (lane == 31) {
    s_wc[w] = ci;
    s_ws[w] = si;
  }
  __syncthreads();
  if (w == 0) {
    unsigned long long x = s_wc[lane];
    double y = s_ws[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long xu = __shfl_up_sync(kFull, x, o);
      const double yu = __shfl_up_sync(kFull, y, o);
      if (lane >= o) {
        x += xu;
        y += yu;
      }
    }
    s_wc[lane] = x;  // inclusive over warps
    s_ws[lane] = y;
  }
  __syncthreads();
  const unsigned long long cw = w ? s_wc[w - 1] : 0ull;
  const double sw = w ? s_ws[w - 1] : 0.0;
  // suffix sums including bin[0] (the higher one) and bin[1]
  const unsigned long long suf1 = cw + ci;  // includes both bins of this thread
  const double ssf1 = sw + si;
  const unsigned long long suf0 = suf1 - c[1];
  const double ssf0 = ssf1 - sm[1];
  const double total_S = s_ws[31];
  const double r = s_st.radius;
  if (level == 1) {
    if (total_S <= r || r <= 0.0) {
      if (tid == 0) {
        L1State st = s_st;
        st.mode = total_S <= r ? 1 : 2;
        st.tau = total_S <= r ? 0.f : INFINITY;
        st.tau_lo = 0.f;
        a.sc->l1[pb] = st;
      }
      return;
    }
  }
  const int pshift = bits + shift;
  const unsigned pre = level == 1 ? 0u : s_st.prefix;
  const unsigned long long suf[2] = {suf0, suf1};
  const double ssf[2] = {ssf0, ssf1};
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    if (bin[e] >= 0) {
      const unsigned lob = (pshift >= 32 ? 0u : (pre << pshift)) | ((unsigned)bin[e] << shift);
      const double lo = (double)__uint_as_float(lob);
      const double h = s_st.S_above + ssf[e] - lo * (double)(s_st.C_above + suf[e]);
      if (h >= r) atomicMax(&s_best, bin[e]);
    }
  }
  __syncthreads();
  int best = s_best;
  if (best < 0) best = 0;  // h(0-edge) >= r holds by construction; guard only
#pragma unroll
  for (int e = 0; e < 2; ++e) {
    if (bin[e] == best) {  // totals strictly above the chosen bin
      s_cx = suf[e] - c[e];
      s_sx = ssf[e] - sm[e];
    }
  }
  __syncthreads();
  if (tid == 0) {
    L1State st = s_st;
    st.C_above += s_cx;
    st.S_above += s_sx;
    st.prefix = (pre << bits) | (unsigned)best;
    if (level == 3) {
      st.mode = 3;
      const double tau = st.C_above > 0 ? (st.S_above - r) / (double)st.C_above : 0.0;
      st.tau = (float)tau;
      st.tau_lo = (float)(tau - (double)st.tau);
    }
    a.sc->l1[pb] = st;
  }
}

// x and out may be the same buffer (an in-place projection): each element is
// read and written by the same thread, and the pointers carry no __restrict__.
__global__ void soft_threshold_kernel(const float *x, float *out, long long n, const Scalars *sc, int prob) {
  const float tau = sc->l1[prob].tau, tau_lo = sc->l1[prob].tau_lo;
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = soft_threshold(x[i], tau, tau_lo);
}

}  // namespace

cudaError_t launch_l1_hist(const L1Args &a, int level, int grid, cudaStream_t st) {
  dim3 g(grid, a.nprob);
  l1_hist_kernel<<<g, 256, 0, st>>>(a, level);
  return cudaGetLastError();
}

cudaError_t launch_l1_scan(const L1Args &a, int level, cudaStream_t st) {
  l1_scan_kernel<<<a.nprob, 1024, 0, st>>>(a, level);
  return cudaGetLastError();
}

cudaError_t launch_soft_threshold(const float *x, float *out, long long n, const Scalars *sc, int prob,
                                  cudaStream_t st) {
  long long g = (n + 255) / 256;
  if (g < 1) g = 1;
  if (g > 4096) g = 4096;
  soft_threshold_kernel<<<(int)g, 256, 0, st>>>(x, out, n, sc, prob);
  return cudaGetLastError();
}

}  // namespace s3ttv
