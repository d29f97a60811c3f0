// Variable-coefficient cylindrical 5-point stencil (Section 2.1, Eqs.
// poisson_diff_2, scheme_op_r_z, diff_approx1, sign-reversed so A > 0):
//
//   (A y)_{i,k} = CR_i (y_{i,k} - y_{i+1,k}) + CR_{i-1} (y_{i,k} - y_{i-1,k})
//               + CZ_{i,k} (y_{i,k} - y_{i,k+1}) + CZ_{i,k-1} (y_{i,k} - y_{i,k-1})
//               + W_{i,k} y_{i,k}
//
// with CR = KR / h_r^2, CZ = KZ / h_z^2 precomputed, CR_0 = 0 on the axis and
// zero values beyond the Dirichlet boundaries r = lr, z = 0, z = lz.
//
// One CTA owns kStencilRows consecutive r-rows and a strip of z-columns of one
// right-hand side.  Each lane holds a short vector (4 FP32 / 2 FP64) of
// consecutive z-nodes and walks down the rows with a three-row register
// window, so every input element is read from memory once (plus one halo row
// per CTA edge).  z-neighbours across lanes come from warp shuffles; the two
// warp-edge lanes fetch one extra element.  blockIdx.x is the right-hand side,
// so CTAs that share a coefficient tile run together and the tile is served
// from L2.
#include "ax_common.cuh"

namespace ax {

namespace {

template <typename T, int MODE>
struct StencilValue {
  // Value of the grid function the operator is applied to, at element e.
  __device__ __forceinline__ static T at(const T *in, const T *p_old, size_t e, T beta) {
    if (MODE == kStencilPcg) return in[e] + beta * p_old[e];
    return in[e];
  }
};

// Hint: bring the line holding p into L2 (no register, no completion; p must
// be a valid global address).
__device__ __forceinline__ void prefetch_l2(const void *p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

template <typename T, int MODE>
__global__ void __launch_bounds__(256) stencil_kernel(const StencilArgs<T> a) {
  constexpr int V = VecT<T>::n;
  __shared__ double red[8];
  const int m = blockIdx.x;
  if (!rhs_selected(a.st, a.mask, m)) return;
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const int k0 = ((blockIdx.z * nwarps + warp) * 32 + lane) * V;
  const int nr = a.nr, nz = a.nz;
  const int i0 = blockIdx.y * kStencilRows;
  const int i1 = min(i0 + kStencilRows, nr);
  const size_t base = (size_t)m * (size_t)a.field;
  const bool col_ok = k0 < nz;
  const T *__restrict__ CR = a.CR + (size_t)m * a.cstride;
  const T *__restrict__ CZ = a.CZ + (size_t)m * a.czstride;
  const T *__restrict__ Wc = a.W + (size_t)m * a.cstride;
  T beta = T(0);
  const T *p_old = nullptr;
  T *p_new = nullptr;
  const T *src = a.in;  // the grid function (before the direction update in mode Pcg)
  if (MODE == kStencilPcg) {
    beta = (T)a.st[m].beta;
    const bool odd = a.st[m].iters & 1;
    p_old = odd ? a.pb : a.pa;
    p_new = odd ? a.pa : a.pb;
  } else if (MODE == kStencilPcgP) {
    src = (a.st[m].iters & 1) ? a.pa : a.pb;
  }

  auto load_row = [&](int i, T (&v)[V]) {
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = T(0);
    if (!col_ok) return;
    const size_t off = base + (size_t)i * a.pitch + k0;
    T t[V];
    load_vec<T>(src + off, t);
    if (MODE == kStencilPcg) {
      T po[V];
      load_vec<T>(p_old + off, po);
#pragma unroll
      for (int e = 0; e < V; ++e) t[e] += beta * po[e];
    }
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = (k0 + e < nz) ? t[e] : T(0);
  };
  auto load_coef = [&](const T *c, int i, T (&v)[V]) {
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = T(0);
    if (!col_ok) return;
    load_vec<T>(c + (size_t)i * a.pitch + k0, v);
  };

  // Everything row i + 1 needs (values, its CR / CZ / W rows and the two
  // warp-edge halo values) is loaded one row ahead, while row i is computed.
  auto load_halo = [&](int i, T &left, T &right, T &czlast) {
    const size_t rowoff = base + (size_t)i * a.pitch;
    left = right = czlast = T(0);
    if (lane == 0 && col_ok && k0 > 0) left = StencilValue<T, MODE>::at(src, p_old, rowoff + k0 - 1, beta);
    if (lane == 31) {
      if (k0 + V < nz) right = StencilValue<T, MODE>::at(src, p_old, rowoff + k0 + V, beta);
      if (k0 + V <= nz) czlast = CZ[(size_t)i * a.pitchz + k0 + V];
    }
  };
  auto load_cz = [&](int i, T (&v)[V]) {
#pragma unroll
    for (int e = 0; e < V; ++e) v[e] = T(0);
    // Faces run to index nz, so the lane just past the last node still loads
    // its first face (the upper face of node nz - 1, fetched by the shuffle).
    if (k0 <= nz) load_vec<T>(CZ + (size_t)i * a.pitchz + k0, v);
  };

  // every row of the DRAM stream(s) this CTA reads, into L2 at once: the
  // register loads below then wait on L2 instead of DRAM
  if (col_ok)
    for (int i = max(i0 - 1, 0); i <= i1 && i < nr; ++i) {
      const size_t off = base + (size_t)i * a.pitch + k0;
      prefetch_l2(src + off);
      if (MODE == kStencilPcg) prefetch_l2(p_old + off);
      if ((MODE == kStencilResidual || MODE == kStencilCheb) && i >= i0 && i < i1) prefetch_l2(a.phi + off);
    }
  T pm[V], pc[V], pn[V], crl[V], crh[V], czl[V], w[V];
  T left, right, czlast;
  if (i0 > 0) {
    load_row(i0 - 1, pm);
    load_coef(CR, i0 - 1, crl);
  } else {
#pragma unroll
    for (int e = 0; e < V; ++e) { pm[e] = T(0); crl[e] = T(0); }
  }
  load_row(i0, pc);
  load_coef(CR, i0, crh);
  load_cz(i0, czl);
  load_coef(Wc, i0, w);
  load_halo(i0, left, right, czlast);

  // FP32 partials per thread are short sums (<= 64 terms); the CTA and grid
  // combination is FP64.
  T acc = T(0);
  for (int i = i0; i < i1; ++i) {
    T crn[V], czn[V], wn[V], leftn = T(0), rightn = T(0), czlastn = T(0);
    if (i + 1 < nr) {
      load_row(i + 1, pn);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) pn[e] = T(0);
    }
    if (i + 1 < i1) {
      load_coef(CR, i + 1, crn);
      load_cz(i + 1, czn);
      load_coef(Wc, i + 1, wn);
      load_halo(i + 1, leftn, rightn, czlastn);
    } else {
#pragma unroll
      for (int e = 0; e < V; ++e) crn[e] = czn[e] = wn[e] = T(0);
    }
    const size_t rowoff = base + (size_t)i * a.pitch;
    // z-neighbours of the lane's first and last node.
    T l = __shfl_up_sync(0xffffffffu, pc[V - 1], 1);
    T r = __shfl_down_sync(0xffffffffu, pc[0], 1);
    T czh_last = __shfl_down_sync(0xffffffffu, czl[0], 1);
    if (lane == 0) l = left;
    if (lane == 31) {
      r = right;
      czh_last = czlast;
    }

    T o[V];
#pragma unroll
    for (int e = 0; e < V; ++e) {
      const T yl = (e == 0) ? l : pc[e - 1];
      const T yr = (e == V - 1) ? r : pc[e + 1];
      const T czh = (e == V - 1) ? czh_last : czl[e + 1];
      const T y = pc[e];
      T v = w[e] * y;
      v = fma(crh[e], y - pn[e], v);
      v = fma(crl[e], y - pm[e], v);
      v = fma(czh, y - yr, v);
      v = fma(czl[e], y - yl, v);
      o[e] = (k0 + e < nz) ? v : T(0);
    }
    if (col_ok) {
      if (MODE == kStencilApply) {
        store_vec<T>(a.out + rowoff + k0, o);
      } else if (MODE == kStencilPcg || MODE == kStencilPcgP) {
        if (MODE == kStencilPcg) store_vec<T>(p_new + rowoff + k0, pc);
        store_vec<T>(a.out + rowoff + k0, o);
#pragma unroll
        for (int e = 0; e < V; ++e) acc = fma(pc[e], o[e], acc);
      } else {
        T ph[V];
        load_vec<T>(a.phi + rowoff + k0, ph);
        T res[V];
#pragma unroll
        for (int e = 0; e < V; ++e) {
          res[e] = (k0 + e < nz) ? ((MODE == kStencilResidual) ? ph[e] - o[e] : o[e] - ph[e]) : T(0);
          acc = fma(res[e], res[e], acc);
        }
        if (MODE == kStencilResidual) {
          if (a.out_res) store_vec<T>(a.out_res + rowoff + k0, res);
          if (a.out32) {
            float r32[4];
#pragma unroll
            for (int e = 0; e < V; ++e) r32[e] = (float)res[e];
            if (V == 4) {
              *reinterpret_cast<float4 *>(a.out32 + rowoff + k0) = make_float4(r32[0], r32[1], r32[2], r32[3]);
            } else {
              *reinterpret_cast<float2 *>(a.out32 + rowoff + k0) = make_float2(r32[0], r32[1]);
            }
          }
        } else {
          store_vec<T>(a.out + rowoff + k0, res);
        }
      }
    }
#pragma unroll
    for (int e = 0; e < V; ++e) {
      pm[e] = pc[e];
      pc[e] = pn[e];
      crl[e] = crh[e];
      crh[e] = crn[e];
      czl[e] = czn[e];
      w[e] = wn[e];
    }
    left = leftn;
    right = rightn;
    czlast = czlastn;
  }
  if (MODE != kStencilApply && a.partial != nullptr) {  // uniform over the CTA
    const double s = block_sum((double)acc, red);
    if (threadIdx.x == 0)
      a.partial[(size_t)m * kPartialStride + blockIdx.y * gridDim.z + blockIdx.z] = s;
  }
}

// ---- double-float residual -------------------------------------------------
// Pairs (h, l) of FP32 numbers carry about 48 significant bits: sums by Knuth's
// two-sum, products by the FMA two-product (the exact error of a*b is
// fma(a, b, -a*b)).  GB300 runs FP32 about 58 times faster than FP64, so the
// true residual of the mixed method costs a few FP32 operations per flop
// instead of FP64 ones.
struct DF {
  float h, l;
};
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return {s, (a - (s - bb)) + (b - bb)};
}

constexpr int kDfRows = 16;      // rows per CTA (short: few right-hand sides are due at a time)
constexpr int kDfThreads = 256;  // 4 z-nodes per thread

__global__ void __launch_bounds__(kDfThreads) residual_df_kernel(const DfResidualArgs a) {
  __shared__ double red[8];
  const int m = blockIdx.z;
  if (!rhs_selected(a.st, a.mask, m)) return;
  const int nr = a.nr, nz = a.nz, P = a.pitch, PZ = a.pitchz;
  const int k0 = (blockIdx.x * kDfThreads + threadIdx.x) * 4;
  const int i0 = blockIdx.y * kDfRows, i1 = min(i0 + kDfRows, nr);
  const bool col_ok = k0 < nz;
  const size_t base = (size_t)m * (size_t)a.field;
  const float *crh = a.CRh + (size_t)m * a.cstride, *crl = a.CRl + (size_t)m * a.cstride;
  const float *czh = a.CZh + (size_t)m * a.czstride, *czl = a.CZl + (size_t)m * a.czstride;
  const float *wh = a.Wh + (size_t)m * a.cstride, *wl = a.Wl + (size_t)m * a.cstride;
  // 4 consecutive values of a field row (zero outside the grid; padding
  // columns hold zeros)
  auto ld4 = [&](const float *p, size_t off, bool ok, float (&v)[4]) {
    if (ok) {
      const float4 t = *reinterpret_cast<const float4 *>(p + off);
      v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    } else {
      v[0] = v[1] = v[2] = v[3] = 0.f;
    }
  };
  float ymh[4], yml[4], ych[4], ycl[4], ynh[4], ynl[4], cph[4], cpl[4];
  ld4(a.xh, base + (size_t)(i0 - 1) * P + k0, col_ok && i0 > 0, ymh);
  ld4(a.xl, base + (size_t)(i0 - 1) * P + k0, col_ok && i0 > 0, yml);
  ld4(crh, (size_t)(i0 - 1) * P + k0, col_ok && i0 > 0, cph);  // CR_{i-1}: 0 on the axis
  ld4(crl, (size_t)(i0 - 1) * P + k0, col_ok && i0 > 0, cpl);
  ld4(a.xh, base + (size_t)i0 * P + k0, col_ok, ych);
  ld4(a.xl, base + (size_t)i0 * P + k0, col_ok, ycl);
  float acc = 0.f;
  for (int i = i0; i < i1; ++i) {
    const size_t ro = (size_t)i * P + k0;
    ld4(a.xh, base + ro + P, col_ok && i + 1 < nr, ynh);
    ld4(a.xl, base + ro + P, col_ok && i + 1 < nr, ynl);
    float cch[4], ccl[4], w4h[4], w4l[4], fh[4], fl[4], zh[4], zl[4];
    ld4(crh, ro, col_ok, cch);
    ld4(crl, ro, col_ok, ccl);
    ld4(wh, ro, col_ok, w4h);
    ld4(wl, ro, col_ok, w4l);
    ld4(a.ph, base + ro, col_ok, fh);
    ld4(a.pl, base + ro, col_ok, fl);
    ld4(czh, (size_t)i * PZ + k0, col_ok, zh);  // faces k0 .. k0 + 3
    ld4(czl, (size_t)i * PZ + k0, col_ok, zl);
    // face k0 + 4 and the z-neighbours outside the 4 nodes
    const bool up_ok = col_ok && k0 + 4 <= nz;
    const DF z4 = {up_ok ? czh[(size_t)i * PZ + k0 + 4] : 0.f, up_ok ? czl[(size_t)i * PZ + k0 + 4] : 0.f};
    const bool left_ok = col_ok && k0 > 0, right_ok = col_ok && k0 + 4 < nz;
    const DF yleft = {left_ok ? a.xh[base + ro - 1] : 0.f, left_ok ? a.xl[base + ro - 1] : 0.f};
    const DF yright = {right_ok ? a.xh[base + ro + 4] : 0.f, right_ok ? a.xl[base + ro + 4] : 0.f};
    float res[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const DF y = {ych[e], ycl[e]};
      const DF yl = (e == 0) ? yleft : DF{ych[e - 1], ycl[e - 1]};
      const DF yr = (e == 3) ? yright : DF{ych[e + 1], ycl[e + 1]};
      const DF czlo = {zh[e], zl[e]};
      const DF czhi = (e == 3) ? z4 : DF{zh[e + 1], zl[e + 1]};
      // r = phi - A y, A y = W y + CR_i (y - y_{i+1}) + CR_{i-1} (y - y_{i-1})
      //                     + CZ_{k+1} (y - y_{k+1}) + CZ_k (y - y_{k-1}),
      // as a compensated sum (Ogita, Rump and Oishi's Dot2: each product's
      // high part exact by the FMA two-product, each addition's error by
      // two-sum, the small terms gathered in one FP32 word): the accuracy of
      // double-float arithmetic without renormalising after every operation
      float sh = fh[e], se = fl[e];
      auto sub_prod = [&](float ch, float cl, float dh, float dl) {  // s -= (ch + cl)(dh + dl)
        const float p = ch * dh;
        const float pe = fmaf(ch, dh, -p);
        const float lo = fmaf(ch, dl, fmaf(cl, dh, pe));
        const float t = sh - p, bb = t - sh;
        se += ((sh - (t - bb)) - (p + bb)) - lo;
        sh = t;
      };
      // y - y_n as an unnormalised pair: the high parts by two-sum, the low
      // parts' difference added to its error
      auto diff = [](DF u, DF w, float &dh, float &dl) {
        const DF s2 = df_two_sum(u.h, -w.h);
        dh = s2.h;
        dl = s2.l + (u.l - w.l);
      };
      float dh, dl;
      sub_prod(w4h[e], w4l[e], y.h, y.l);
      diff(y, DF{ynh[e], ynl[e]}, dh, dl);
      sub_prod(cch[e], ccl[e], dh, dl);
      diff(y, DF{ymh[e], yml[e]}, dh, dl);
      sub_prod(cph[e], cpl[e], dh, dl);
      diff(y, yr, dh, dl);
      sub_prod(czhi.h, czhi.l, dh, dl);
      diff(y, yl, dh, dl);
      sub_prod(czlo.h, czlo.l, dh, dl);
      res[e] = (k0 + e < nz) ? sh + se : 0.f;
      acc = fmaf(res[e], res[e], acc);
    }
    if (col_ok) *reinterpret_cast<float4 *>(a.r32 + base + ro) = make_float4(res[0], res[1], res[2], res[3]);
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      ymh[e] = ych[e]; yml[e] = ycl[e];
      ych[e] = ynh[e]; ycl[e] = ynl[e];
      cph[e] = cch[e]; cpl[e] = ccl[e];
    }
  }
  const double sum = block_sum((double)acc, red);
  if (threadIdx.x == 0) a.partial[(size_t)m * kPartialStride + blockIdx.y * gridDim.x + blockIdx.x] = sum;
}

int column_warps(int nz, int vec) {
  int w = (nz + 32 * vec - 1) / (32 * vec);
  return w < kStencilWarps ? (w < 1 ? 1 : w) : kStencilWarps;
}

}  // namespace

int stencil_blocks_per_rhs(int nr, int nz, int vec) {
  const int wx = column_warps(nz, vec);
  const int gz = (nz + 32 * vec * wx - 1) / (32 * vec * wx);
  const int gy = (nr + kStencilRows - 1) / kStencilRows;
  return gy * gz;
}

template <typename T>
void launch_stencil(int mode, const StencilArgs<T> &a, cudaStream_t s) {
  constexpr int V = VecT<T>::n;
  const int wx = column_warps(a.nz, V);
  dim3 grid(a.m, (a.nr + kStencilRows - 1) / kStencilRows, (a.nz + 32 * V * wx - 1) / (32 * V * wx));
  dim3 block(32 * wx);
  note_launch();
  switch (mode) {
    case kStencilApply: stencil_kernel<T, kStencilApply><<<grid, block, 0, s>>>(a); break;
    case kStencilPcg: stencil_kernel<T, kStencilPcg><<<grid, block, 0, s>>>(a); break;
    case kStencilPcgP: stencil_kernel<T, kStencilPcgP><<<grid, block, 0, s>>>(a); break;
    case kStencilResidual: stencil_kernel<T, kStencilResidual><<<grid, block, 0, s>>>(a); break;
    default: stencil_kernel<T, kStencilCheb><<<grid, block, 0, s>>>(a); break;
  }
}

int residual_df_blocks(int nr, int nz) {
  return ((nz + 4 * kDfThreads - 1) / (4 * kDfThreads)) * ((nr + kDfRows - 1) / kDfRows);
}

void launch_residual_df(const DfResidualArgs &a, cudaStream_t s) {
  dim3 grid((a.nz + 4 * kDfThreads - 1) / (4 * kDfThreads), (a.nr + kDfRows - 1) / kDfRows, a.m);
  note_launch();
  residual_df_kernel<<<grid, kDfThreads, 0, s>>>(a);
}

template void launch_stencil<float>(int, const StencilArgs<float> &, cudaStream_t);
template void launch_stencil<double>(int, const StencilArgs<double> &, cudaStream_t);

}  // namespace ax
