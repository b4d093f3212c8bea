// Compute for the compute-plus-communication demonstration: one Jacobi sweep over a
// subdomain with halo rows, the workload of the paper's application study (Sec. 5.4: a
// Jacobi solver whose subdomains exchange boundary rows with their two neighbours, a ring).
// The paper puts only the transfers into CUDA graphs and expects larger gains once kernels
// join them; this kernel lets a caller capture stencil sweeps and multi-path halo
// exchanges into one graph.
//
// Layout: (rows + 2) x cols fp32, row-major, row 0 and row rows+1 the halos.  For interior
// rows r and columns 1..cols-2:
//   out[r][c] = ((in[r-1][c] + in[r+1][c]) + (in[r][c-1] + in[r][c+1])) * 0.25
// in that operation order, each step rounded to fp32 (so a CPU program in the same order
// reproduces it bit for bit); columns 0 and cols-1 are copied unchanged; halo rows of
// `out` are not written.
#include "internal.h"

namespace mpt {
namespace {

__global__ void __launch_bounds__(256) k_jacobi(const float* __restrict__ in, float* __restrict__ out, uint32_t rows,
                                              uint64_t cols) {
  const uint64_t total = (uint64_t)rows * cols;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t r = i / cols + 1, c = i % cols;
    const float* row = in + r * cols;
    float v;
    if (c == 0 || c + 1 == cols) {
      v = row[c];
    } else {
      const float vert = __fadd_rn(row[c - cols], row[c + cols]);
      const float horiz = __fadd_rn(row[c - 1], row[c + 1]);
      v = __fmul_rn(__fadd_rn(vert, horiz), 0.25f);
    }
    out[r * cols + c] = v;
  }
}

}  // namespace
}  // namespace mpt

extern "C" MPT_API mpt_status mpt_demo_jacobi_step(const float* in, float* out, uint32_t rows, uint64_t cols,
                                                   void* stream) {
  if (!in || !out || rows == 0 || cols < 2) return mpt::fail(MPT_EINVAL, "mpt_demo_jacobi_step: bad argument");
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return mpt::fail(MPT_ECUDA, "mpt_demo_jacobi_step: device query");
  const uint64_t total = (uint64_t)rows * cols;
  const uint64_t want = (total + 255) / 256;
  const uint32_t blocks = (uint32_t)(want < 8ull * sms ? (want ? want : 1) : 8ull * sms);
  mpt::k_jacobi<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(in, out, rows, cols);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mpt::fail(MPT_ECUDA, "mpt_demo_jacobi_step: %s", cudaGetErrorString(e));
  return MPT_OK;
}
