// runtime.cu -- host-side plumbing: thread-local error text, device
// properties, and the tensor-map encoder (driver entry point fetched through
// the runtime, so the library does not link libcuda directly).
#include <mutex>
#include <string>

#include "internal.h"

namespace sks {

namespace {
thread_local std::string g_last_error;

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
}  // namespace

void set_last_error(const std::string& msg) { g_last_error = msg; }

sks_status fail(sks_status code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

const char* last_error_cstr() { return g_last_error.c_str(); }

namespace {
thread_local uint64_t g_launches = 0;
}
void note_launch(int count) { g_launches += (uint64_t)count; }
uint64_t launch_count() { return g_launches; }

const DeviceInfo& device_info() {
  static thread_local DeviceInfo info;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return info;
  if (info.device != dev) {
    info.device = dev;
    cudaDeviceGetAttribute(&info.sms, cudaDevAttrMultiProcessorCount, dev);
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    info.smem_optin = (size_t)optin;
  }
  return info;
}

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

sks_status make_tmap_2d_bf16_sw128(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols,
                                   uint32_t box_cols, uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(SKS_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
  if (((uintptr_t)base & 127) != 0) return fail(SKS_ERR_INVALID_ARG, "bf16 operand must be 128-byte aligned");
  if ((cols * 2) % 16 != 0 || box_cols * 2 != 128) return fail(SKS_ERR_INVALID_ARG, "bf16 tensor map geometry");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)(rows > 0 ? rows : 1)};
  cuuint64_t strides[1] = {(cuuint64_t)(cols * 2)};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(SKS_ERR_INVALID_ARG, "cuTensorMapEncodeTiled (bf16) failed (code " + std::to_string((int)r) + ")");
  return SKS_OK;
}

sks_status make_tmap_2d_u8_sw128(CUtensorMap* map, const void* base, uint64_t rows, uint64_t cols, uint32_t box_cols,
                                 uint32_t box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return fail(SKS_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
  if (((uintptr_t)base & 127) != 0) return fail(SKS_ERR_INVALID_ARG, "8-bit operand must be 128-byte aligned");
  if (cols % 16 != 0 || box_cols != 128) return fail(SKS_ERR_INVALID_ARG, "8-bit tensor map geometry");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)(rows > 0 ? rows : 1)};
  cuuint64_t strides[1] = {(cuuint64_t)cols};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS)
    return fail(SKS_ERR_INVALID_ARG, "cuTensorMapEncodeTiled (8-bit) failed (code " + std::to_string((int)r) + ")");
  return SKS_OK;
}

sks_status make_tmap_2d(CUtensorMap* map, const void* base, CUtensorMapDataType dt, size_t elem_bytes, uint64_t rows,
                        uint64_t cols, uint64_t ld, uint32_t box_cols, uint32_t box_rows) {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  static cudaError_t qerr = cudaSuccess;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    qerr = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q);
    if (qerr == cudaSuccess && q == cudaDriverEntryPointSuccess) fn = (EncodeTiledFn)p;
  });
  if (!fn) return fail(SKS_ERR_CUDA, "cuTensorMapEncodeTiled entry point unavailable");
  if (((uintptr_t)base & 15) != 0) return fail(SKS_ERR_INVALID_ARG, "A must be 16-byte aligned");
  if ((ld * elem_bytes) % 16 != 0) return fail(SKS_ERR_INVALID_ARG, "lda * element size must be a multiple of 16 bytes");
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)(rows > 0 ? rows : 1)};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * elem_bytes)};
  cuuint32_t box[2] = {box_cols, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return fail(SKS_ERR_INVALID_ARG, "cuTensorMapEncodeTiled failed (code " + std::to_string((int)r) + ")");
  return SKS_OK;
}

// ---------------------------------------------------------------- failure-path self-test
namespace {
__device__ DevStatus g_selftest_status;

// One thread waits on an mbarrier that nothing ever arrives on; the bounded
// wait gives up after limit_ns and records SKS_ERR_TIMEOUT.
__global__ void selftest_wait_kernel(DevStatus* st, uint64_t limit_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    fence_mbar_init();
  }
  __syncthreads();
  if (threadIdx.x == 0) mbar_wait(&bar, 0u, st, 99, limit_ns);
}
}  // namespace

sks_status selftest_wait_timeout(long long limit_ns, cudaStream_t stream) {
  if (limit_ns < 1000 || limit_ns > 1000000000ll) return fail(SKS_ERR_INVALID_ARG, "limit_ns must be in [1e3, 1e9]");
  DevStatus* st = nullptr;
  SKS_CUDA_TRY(cudaGetSymbolAddress((void**)&st, g_selftest_status));
  SKS_CUDA_TRY(cudaMemsetAsync(st, 0, sizeof(DevStatus), stream));
  selftest_wait_kernel<<<1, 32, 0, stream>>>(st, (uint64_t)limit_ns);
  note_launch();
  SKS_CUDA_TRY(cudaGetLastError());
  return read_status(st, stream, "self-test wait");
}

}  // namespace sks
