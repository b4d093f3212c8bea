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

__device__ __forceinline__ float jacobi_point(float up, float down, float left, float right) {
  return __fmul_rn(__fadd_rn(__fadd_rn(up, down), __fadd_rn(left, right)), 0.25f);
}

__device__ __forceinline__ float4 ld4(const float4* p) { return __ldg(p); }

// Column-strip sweep: thread q owns columns 4q..4q+3 (one float4) of every row and walks
// down the rows with the rows above, at and below the current one in registers (the next
// one already in flight), so each input row is read once and each output row written once.
// Horizontal neighbours come from the adjacent lanes (warp shuffles); the two lanes at a
// warp's edges read their outside neighbour from global memory.  Needs cols % 4 == 0 and
// 16-byte aligned rows.
__global__ void __launch_bounds__(256) k_jacobi_v4(const float* __restrict__ in, float* __restrict__ out,
                                                  uint32_t rows, uint64_t cols) {
  const uint64_t nq = cols / 4;
  const uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool active = q < nq;
  const uint64_t qq = active ? q : nq - 1;  // idle lanes shadow the last quad (shuffles need them)
  const uint32_t lane = threadIdx.x & 31u;
  const uint64_t c0 = 4 * qq;
  const float4* in4 = reinterpret_cast<const float4*>(in);
  float4* out4 = reinterpret_cast<float4*>(out);
  float4 up = ld4(in4 + qq), mid = ld4(in4 + nq + qq), down = ld4(in4 + 2 * nq + qq);
  for (uint32_t r = 1; r <= rows; ++r) {
    const float4 next = (r + 2 <= rows + 1) ? ld4(in4 + (uint64_t)(r + 2) * nq + qq) : down;
    float left = __shfl_up_sync(0xffffffffu, mid.w, 1);
    float right = __shfl_down_sync(0xffffffffu, mid.x, 1);
    const float* row = in + (uint64_t)r * cols;
    if (lane == 0 && c0 > 0) left = row[c0 - 1];
    if (lane == 31 && c0 + 4 < cols) right = row[c0 + 4];
    // (a quad whose right neighbour lies past the row ends in column cols-1, copied as is)
    float4 o;
    o.x = c0 == 0 ? mid.x : jacobi_point(up.x, down.x, left, mid.y);
    o.y = jacobi_point(up.y, down.y, mid.x, mid.z);
    o.z = jacobi_point(up.z, down.z, mid.y, mid.w);
    o.w = c0 + 4 == cols ? mid.w : jacobi_point(up.w, down.w, mid.z, right);
    if (active) out4[(uint64_t)r * nq + q] = o;
    up = mid;
    mid = down;
    down = next;
  }
}

// Any column count or alignment: one thread per point, rows over blockIdx.y (strided).
__global__ void __launch_bounds__(256) k_jacobi(const float* __restrict__ in, float* __restrict__ out, uint32_t rows,
                                              uint64_t cols) {
  const uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  for (uint32_t r = 1 + blockIdx.y; r <= rows; r += gridDim.y) {
    const float* row = in + (uint64_t)r * cols;
    float v;
    if (c == 0 || c + 1 == cols) {
      v = row[c];
    } else {
      v = jacobi_point(row[c - cols], row[c + cols], row[c - 1], row[c + 1]);
    }
    out[(uint64_t)r * cols + c] = v;
  }
}

}  // namespace
}  // namespace mpt

extern "C" MPT_API mpt_status mpt_demo_jacobi_step(const float* in, float* out, uint32_t rows, uint64_t cols,
                                                   void* stream) {
  if (!in || !out || rows == 0 || cols < 2) return mpt::fail(MPT_EINVAL, "mpt_demo_jacobi_step: bad argument");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const bool vec = cols % 4 == 0 && (reinterpret_cast<uintptr_t>(in) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(out) & 15) == 0;
  if (vec) {
    const uint64_t blocks = (cols / 4 + 255) / 256;
    if (blocks > 0x7fffffffull) return mpt::fail(MPT_EINVAL, "mpt_demo_jacobi_step: %llu columns", (unsigned long long)cols);
    mpt::k_jacobi_v4<<<(uint32_t)blocks, 256, 0, s>>>(in, out, rows, cols);
  } else {
    const uint64_t bx = (cols + 255) / 256;
    if (bx > 0x7fffffffull) return mpt::fail(MPT_EINVAL, "mpt_demo_jacobi_step: %llu columns", (unsigned long long)cols);
    const uint32_t by = rows < 65535u ? rows : 65535u;
    mpt::k_jacobi<<<dim3((uint32_t)bx, by), 256, 0, s>>>(in, out, rows, cols);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return mpt::fail(MPT_ECUDA, "mpt_demo_jacobi_step: %s", cudaGetErrorString(e));
  return MPT_OK;
}
