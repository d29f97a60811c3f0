// Preconditioner application that allocates no device memory.
//
// ax_apply_preconditioner stages its input in a workspace that the operator
// grows with cudaMalloc on first use.  Some callers cannot allow that: code
// running while a stream is being captured into a CUDA graph, allocators that
// own all device memory, or real-time loops that must not call into the
// memory manager.  This entry point does the same work (sine transform, mode
// solves, inverse transform) but stages through one fixed array compiled
// into the library instead.
//
// Facts a caller must know:
//  * The array holds kNoAllocScratchBytes (32 MiB) on every GPU that loads the
//    library, from module load until process exit.
//  * One call needs 2 * m * nr * pitch * sizeof(T) bytes of it (pitch = nz
//    rounded up to 32, T = double or float by precision); larger requests are
//    refused with AX_ERR_INVALID_ARG before any work is queued.
//  * The first call on a device looks up the array's device address
//    (cudaGetSymbolAddress) with that device current; make that first call
//    before any stream capture begins.  Later calls only queue kernels.
//  * All calls share the one array, and it keeps the last call's contents.
//    Each call writes every element it later reads (the packing pass also
//    zeroes the padding columns of both halves), so no clearing is needed.
//    Two calls whose work
//    overlaps on the GPU (different streams, no ordering between them) race
//    on the array and corrupt each other's results: order them.
#include <cmath>
#include <mutex>

#include "ax_common.cuh"

namespace ax {
namespace {

constexpr size_t kNoAllocScratchBytes = 32ull << 20;
constexpr int kMaxDevices = 64;

// Device-side scratch.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void *g_noalloc_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device (looked up once
// per device).  Returns AX_OK or an error status.
int noalloc_scratch(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return AX_ERR_CUDA;
  if (dev < 0 || dev >= kMaxDevices) return AX_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr) return AX_ERR_CUDA;
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return AX_OK;
}

// Packs the dense input rows into the padded layout of the first half and
// zeroes the padding columns nz .. pitch-1 of both halves: the transforms'
// vector loads cover those columns, and the array keeps the previous call's
// contents.
template <typename T>
__global__ void noalloc_pack(const double *__restrict__ src, T *__restrict__ dst, T *__restrict__ dst2,
                             long long rows, int nz, int pitch) {
  for (long long row = blockIdx.x; row < rows; row += gridDim.x)
    for (int k = threadIdx.x; k < pitch; k += blockDim.x) {
      dst[row * pitch + k] = k < nz ? (T)src[row * nz + k] : T(0);
      if (k >= nz) dst2[row * pitch + k] = T(0);
    }
}

template <typename T>
__global__ void noalloc_unpack(const T *__restrict__ src, double *__restrict__ dst, long long rows, int nz,
                               int pitch) {
  for (long long row = blockIdx.x; row < rows; row += gridDim.x)
    for (int k = threadIdx.x; k < nz; k += blockDim.x) dst[row * nz + k] = (double)src[row * pitch + k];
}

template <typename T> const Coef<T> &coef_of(const ax_operator *op);
template <> const Coef<double> &coef_of<double>(const ax_operator *op) { return op->c64; }
template <> const Coef<float> &coef_of<float>(const ax_operator *op) { return op->c32; }

template <typename T>
int precond_noalloc(ax_operator *op, const double *in, double *out, int m, cudaStream_t s) {
  const size_t field = (size_t)op->nr * op->pitch;
  const size_t need = 2 * field * (size_t)m * sizeof(T);
  if (need > kNoAllocScratchBytes) return AX_ERR_INVALID_ARG;
  void *base = nullptr;
  int rc = noalloc_scratch(&base);
  if (rc != AX_OK) return rc;
  T *a = reinterpret_cast<T *>(base);
  T *b = a + field * m;
  const Coef<T> &c = coef_of<T>(op);
  const long long rows = (long long)op->nr * m;
  const int blocks = (int)(rows < 65535 ? rows : 65535);

  note_launch();
  noalloc_pack<T><<<blocks, 256, 0, s>>>(in, a, b, rows, op->nz, op->pitch);

  DstArgs<T> d{};
  d.TW = c.TW;
  d.HW = c.HW;
  d.CW = c.CW;
  d.cosine = op->bc_z == 1;
  d.RK = c.RK;
  d.RT = c.RT;
  d.RP = op->rader_perm;
  d.plan = op->plan;
  d.n = op->nz;
  d.rows = op->nr;
  d.pitch = op->pitch;
  d.field = (long long)field;
  d.m = m;
  d.scale = op->bc_z == 1 ? 1.0 / std::sqrt(2.0 * op->nz) : 0.5 / std::sqrt(2.0 * op->plan.L);
  d.st = nullptr;
  d.mask = -1;
  d.in = a;
  d.out = b;
  launch_dst<T>(kDstPlain, d, s);

  TriArgs<T> t{};
  t.IP = c.IP;
  t.E = c.E;
  t.cstride = op->cstride;
  t.estride = op->estride;
  t.nr = op->nr;
  t.nz = op->nz;
  t.pitch = op->pitch;
  t.field = (long long)field;
  t.m = m;
  t.in = b;
  t.out = b;
  t.st = nullptr;
  t.mask = -1;
  launch_tridiag<T>(t, s);

  d.in = b;
  d.out = b;
  d.inverse = 1;
  launch_dst<T>(kDstPlain, d, s);

  note_launch();
  noalloc_unpack<T><<<blocks, 256, 0, s>>>(b, out, rows, op->nz, op->pitch);
  return cudaGetLastError() == cudaSuccess ? AX_OK : AX_ERR_CUDA;
}

}  // namespace
}  // namespace ax

extern "C" int ax_apply_preconditioner_noalloc(ax_operator *op, const double *in, double *out, int32_t m,
                                               int32_t precision, void *stream) {
  if (!op || !in || !out || m < 1) return AX_ERR_INVALID_ARG;
  if (precision != AX_PREC_FP64 && precision != AX_PREC_FP32) return AX_ERR_INVALID_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  return precision == AX_PREC_FP64 ? ax::precond_noalloc<double>(op, in, out, m, s)
                                   : ax::precond_noalloc<float>(op, in, out, m, s);
}
