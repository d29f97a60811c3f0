// Sine and cosine transforms, FP32 instantiation (see ax_dst_impl.cuh).
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

int dst_rows_per_block(int L, int elem_bytes) {
  const size_t per_row = 2ull * L * 2 * elem_bytes;
  size_t r = (kDstSmemBudget - 4 * elem_bytes) / per_row;
  if (r < 1) r = 1;
  if (r > 16) r = 16;
  return (int)r;
}

size_t dst_smem_bytes(int L, int elem_bytes) {
  // two buffers of rpb rows of L complex values; the second starts on a
  // 16-byte boundary (one complex of slack)
  return ((size_t)dst_rows_per_block(L, elem_bytes) * L + 1) * 2ull * 2 * elem_bytes;
}

int dst_prepare_f32() { return fill_prime_table<float>(c_prime_f); }

int dst_prepare_device() {
  static bool done[64] = {false};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return AX_ERR_CUDA;
  if (done[dev]) return AX_OK;
  int rc = dst_prepare_f32();
  if (rc == AX_OK) rc = dst_prepare_f64();
  if (rc == AX_OK) done[dev] = true;
  return rc;
}

template <>
void launch_dst<float>(int mode, const DstArgs<float> &a, cudaStream_t s) {
  launch_dst_any<float>(mode, a, s);
}

}  // namespace ax
