// Small HBM-bound helper kernels: the k == 0 epilogue (C = beta * C_in) and
// per-tensor FP8 E4M3 quantisation.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include <algorithm>
#include <cstring>

#include "common.cuh"

namespace sk {

namespace {

template <typename T>
__global__ void scale_kernel(T *C, const T *C_in, int64_t ldc, int64_t M, int64_t N, float beta) {
  const int64_t total = M * N;
  for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = idx / N, j = idx - (idx / N) * N;
    float v = 0.f;
    if (beta != 0.f) v = beta * static_cast<float>(C_in[i * ldc + j]);
    C[i * ldc + j] = static_cast<T>(v);
  }
}

// amax over |x| as the bit pattern of a non-negative float (monotone in the
// value, so an unsigned atomicMax is exact).  NaNs are ignored.
__global__ void amax_kernel(const float *x, int64_t n, unsigned int *amax_bits) {
  float m = 0.f;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  __shared__ float wmax[32];
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    m = threadIdx.x < (blockDim.x >> 5) ? wmax[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (threadIdx.x == 0) atomicMax(amax_bits, __float_as_uint(m));
  }
}

// scale = amax / 448 (1 if amax == 0); q = E4M3(x / scale), round to nearest
// even, saturating to +-448 (satfinite conversion).
__global__ void quant_kernel(const float *x, int64_t n, uint8_t *q, float *scale_out, const float *amax) {
  const float a = *amax;
  const float s = a > 0.f ? __fdiv_rn(a, 448.0f) : 1.0f;
  if (blockIdx.x == 0 && threadIdx.x == 0) *scale_out = s;
  const int64_t pairs = n / 2;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < pairs; i += (int64_t)gridDim.x * blockDim.x) {
    float2 v = reinterpret_cast<const float2 *>(x)[i];
    v.x = __fdiv_rn(v.x, s);
    v.y = __fdiv_rn(v.y, s);
    __nv_fp8x2_storage_t r = __nv_cvt_float2_to_fp8x2(v, __NV_SATFINITE, __NV_E4M3);
    reinterpret_cast<__nv_fp8x2_storage_t *>(q)[i] = r;
  }
  if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) {
    q[n - 1] = __nv_cvt_float_to_fp8(__fdiv_rn(x[n - 1], s), __NV_SATFINITE, __NV_E4M3);
  }
}

// dst = transpose of src for 16-bit elements: src is rows x cols row-major
// (leading dimension ld_src), dst cols x rows row-major (ld_dst).  64 x 64
// tiles through shared memory (row pitch 66 elements: a column gather hits
// each bank at most twice), 16-byte global loads and stores where a group of
// 8 elements lies inside the matrix and both row pitches are multiples of 8
// elements (the caller's 16-byte-aligned operands), element by element at the
// ragged edges.  A grid-stride loop over tiles keeps any size in one launch;
// each thread loads its part of the next tile into registers before it
// gathers and stores the current one, so a tile's load latency overlaps the
// previous tile's stores.
__global__ void __launch_bounds__(256) transpose16_kernel(const uint16_t *__restrict__ src, int64_t rows, int64_t cols,
                                                          int64_t ld_src, uint16_t *__restrict__ dst, int64_t ld_dst,
                                                          int vec) {
  __shared__ __align__(16) uint16_t tile[64][66];
  const int64_t tr = (rows + 63) / 64, tc = (cols + 63) / 64, ntiles = tr * tc;
  const int t = threadIdx.x;
  uint16_t v[2][8];
  auto load = [&](int64_t tile_id) {
    const int64_t r0 = (tile_id / tc) * 64, c0 = (tile_id % tc) * 64;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int64_t gr = r0 + t / 8 + 32 * p, gc = c0 + 8 * (t % 8);
      if (vec && gr < rows && gc + 8 <= cols) {
        const uint4 q = __ldcs(reinterpret_cast<const uint4 *>(src + gr * ld_src + gc));
        std::memcpy(v[p], &q, 16);
      } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) v[p][e] = (gr < rows && gc + e < cols) ? src[gr * ld_src + gc + e] : (uint16_t)0;
      }
    }
  };
  int64_t tile_id = blockIdx.x;
  if (tile_id < ntiles) load(tile_id);
  for (; tile_id < ntiles; tile_id += gridDim.x) {
    const int64_t r0 = (tile_id / tc) * 64, c0 = (tile_id % tc) * 64;
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int r = t / 8 + 32 * p, c = 8 * (t % 8);
#pragma unroll
      for (int e = 0; e < 8; e += 2)
        *reinterpret_cast<uint32_t *>(&tile[r][c + e]) = (uint32_t)v[p][e] | ((uint32_t)v[p][e + 1] << 16);
    }
    __syncthreads();
    if (tile_id + gridDim.x < ntiles) load(tile_id + gridDim.x);   // in flight during the stores below
#pragma unroll
    for (int p = 0; p < 2; ++p) {
      const int j = t / 8 + 32 * p, i = 8 * (t % 8);   // dst row j (src column), dst columns i .. i+7
      const int64_t gr = c0 + j, gc = r0 + i;
      if (gr < cols) {
        uint16_t w[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) w[e] = tile[i + e][j];
        if (vec && gc + 8 <= rows) {
          uint4 q;
          std::memcpy(&q, w, 16);
          __stcs(reinterpret_cast<uint4 *>(dst + gr * ld_dst + gc), q);
        } else {
#pragma unroll
          for (int e = 0; e < 8; ++e)
            if (gc + e < rows) dst[gr * ld_dst + gc + e] = w[e];
        }
      }
    }
    __syncthreads();
  }
}

struct UploadBlock {
  uint4 *dst;
  uint32_t n16;   // 16-byte words carried
  uint32_t pad_;
  uint4 data[UPLOAD_CHUNK_BYTES / 16];
};

__global__ void upload_kernel(const __grid_constant__ UploadBlock b) {
  for (uint32_t i = threadIdx.x; i < b.n16; i += blockDim.x) b.dst[i] = b.data[i];
  // the words may hold tensor maps that later kernels hand to the TMA unit
  asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
}

}  // namespace

cudaError_t launch_transpose16(const void *src, int64_t rows, int64_t cols, int64_t ld_src, void *dst, int64_t ld_dst,
                               int sms, cudaStream_t st) {
  if (rows <= 0 || cols <= 0) return cudaSuccess;
  const int vec = (reinterpret_cast<uintptr_t>(src) & 15u) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15u) == 0 &&
                  ld_src % 8 == 0 && ld_dst % 8 == 0;
  const int64_t tiles = ((rows + 63) / 64) * ((cols + 63) / 64);
  const int grid = (int)std::min<int64_t>(tiles, (int64_t)std::max(1, sms) * 8);
  transpose16_kernel<<<grid, 256, 0, st>>>(static_cast<const uint16_t *>(src), rows, cols, ld_src,
                                           static_cast<uint16_t *>(dst), ld_dst, vec);
  return cudaGetLastError();
}

cudaError_t launch_upload(void *dst, const void *src, size_t bytes, cudaStream_t st) {
  if ((bytes & 15u) || (reinterpret_cast<uintptr_t>(dst) & 15u)) return cudaErrorInvalidValue;
  const uint8_t *s = static_cast<const uint8_t *>(src);
  uint8_t *d = static_cast<uint8_t *>(dst);
  UploadBlock *b = new UploadBlock();
  cudaError_t e = cudaSuccess;
  for (size_t off = 0; off < bytes && e == cudaSuccess; off += UPLOAD_CHUNK_BYTES) {
    const size_t n = bytes - off < (size_t)UPLOAD_CHUNK_BYTES ? bytes - off : (size_t)UPLOAD_CHUNK_BYTES;
    b->dst = reinterpret_cast<uint4 *>(d + off);
    b->n16 = (uint32_t)(n / 16);
    b->pad_ = 0;
    std::memcpy(b->data, s + off, n);
    upload_kernel<<<1, 256, 0, st>>>(*b);
    e = cudaGetLastError();
  }
  delete b;
  return e;
}

cudaError_t launch_scale(void *C, const void *C_in, int64_t ldc, int64_t M, int64_t N, float beta, int c_is_f32,
                         cudaStream_t st) {
  const int64_t total = M * N;
  int blocks = (int)((total + 255) / 256);
  if (blocks > 4096) blocks = 4096;
  if (blocks < 1) blocks = 1;
  if (c_is_f32)
    scale_kernel<float><<<blocks, 256, 0, st>>>(static_cast<float *>(C), static_cast<const float *>(C_in), ldc, M, N,
                                                beta);
  else
    scale_kernel<__nv_bfloat16><<<blocks, 256, 0, st>>>(static_cast<__nv_bfloat16 *>(C),
                                                        static_cast<const __nv_bfloat16 *>(C_in), ldc, M, N, beta);
  return cudaGetLastError();
}

cudaError_t launch_quant_e4m3(const float *x, int64_t n, uint8_t *q, float *scale_out, float *amax_work,
                              cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(amax_work, 0, sizeof(float), st);
  if (e != cudaSuccess) return e;
  int blocks = (int)((n + 1023) / 1024);
  if (blocks > 2048) blocks = 2048;
  if (blocks < 1) blocks = 1;
  amax_kernel<<<blocks, 256, 0, st>>>(x, n, reinterpret_cast<unsigned int *>(amax_work));
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  quant_kernel<<<blocks, 256, 0, st>>>(x, n, q, scale_out, amax_work);
  return cudaGetLastError();
}

}  // namespace sk
