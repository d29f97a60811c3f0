// Sine and cosine transforms, FP64 instantiation (see ax_dst_impl.cuh).
#include "ax_dst_impl.cuh"

namespace ax {
namespace {
template <typename T>
void launch_dst_any(int mode, const DstArgs<T> &a_in, cudaStream_t s) {
  DstArgs<T> a = a_in;
  const int LB = dst_buffer_len(a.plan.L, a.n);
  a.rpb = dst_rows_per_block(LB, (int)sizeof(T));
  size_t smem = dst_smem_bytes(LB, (int)sizeof(T));
  if (a.plan.rader) smem += 2ull * a.rpb * a.plan.tn_div[0].d * 2 * sizeof(T);
  dim3 grid(a.m, (a.rows + a.rpb - 1) / a.rpb);
  dim3 block(256);
  note_launch();
  switch (mode) {
    case kDstPlain:
      ensure_smem_attr((const void *)dst_kernel<T, kDstPlain>, smem);
      dst_kernel<T, kDstPlain><<<grid, block, smem, s>>>(a);
      break;
    case kDstPcgForward:
      ensure_smem_attr((const void *)dst_kernel<T, kDstPcgForward>, smem);
      dst_kernel<T, kDstPcgForward><<<grid, block, smem, s>>>(a);
      break;
    case kDstPcgInverse:
      ensure_smem_attr((const void *)dst_kernel<T, kDstPcgInverse>, smem);
      dst_kernel<T, kDstPcgInverse><<<grid, block, smem, s>>>(a);
      break;
    default:
      ensure_smem_attr((const void *)dst_kernel<T, kDstChebInverse>, smem);
      dst_kernel<T, kDstChebInverse><<<grid, block, smem, s>>>(a);
      break;
  }
}

// Fills this translation unit's table of cos / sin(2 pi j / R).
template <typename T, size_t N>
int fill_prime_table(const T (&sym)[N]) {
  T h[N];
  for (int i = 0, off = 0; i < kNumUnrolled; ++i) {
    const int R = kUnrolledPrimes[i];
    for (int j = 0; j < R; ++j) {
      h[off + 2 * j] = (T)std::cos(2.0 * M_PI * j / R);
      h[off + 2 * j + 1] = (T)std::sin(2.0 * M_PI * j / R);
    }
    off += 2 * R;
  }
  return cudaMemcpyToSymbol(sym, h, sizeof(h)) == cudaSuccess ? AX_OK : AX_ERR_CUDA;
}
}  // namespace

int dst_prepare_f64() { return fill_prime_table<double>(c_prime_d); }

template <>
void launch_dst<double>(int mode, const DstArgs<double> &a, cudaStream_t s) {
  launch_dst_any<double>(mode, a, s);
}

}  // namespace ax
