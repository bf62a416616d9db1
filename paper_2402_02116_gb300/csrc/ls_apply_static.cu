// ls_apply_noalloc: the LS operator pass of ls_apply with its scratch space in a fixed device array
// of this library instead of a caller-supplied work buffer.
//
// Some callers cannot hand the library a work buffer: code that is not allowed to allocate device
// memory once it is running (a plugin whose host application owns every device allocation, a
// loop with a fixed memory budget set at start-up) still needs the operator. For them the
// scratch lives in `g_scratch` below, a file-scope device array of kStaticScratchBytes that every
// GPU loading this library keeps until the process exits. The entry point allocates and frees
// nothing: it looks up the array's device address, checks that the batch fits, and runs the same
// kernels as ls_apply on that memory.
#include <mutex>

#include "common.cuh"

namespace dbi {

// 32 MiB: e.g. 15 problems of 256 x 256 cells on a 512 x 512 FFT grid in complex64.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;

static __device__ __align__(256) unsigned char g_scratch[kStaticScratchBytes];

// Device address of g_scratch for each device, looked up once with that device current. In host
// code `g_scratch` names a host-side shadow, not device memory, so it must never be passed to a
// kernel directly.
constexpr int kMaxDevices = 64;
static void *g_scratch_ptr[kMaxDevices] = {};
static std::mutex g_scratch_mu;

static int scratch_address(void **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail("cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d is beyond the %d devices ls_apply_noalloc supports", dev, kMaxDevices);
    return DBI_ERR_UNSUPPORTED;
  }
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return cuda_fail("cudaGetSymbolAddress(g_scratch)", e);
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return DBI_OK;
}

}  // namespace dbi

using namespace dbi;

extern "C" size_t dbi_noalloc_scratch_bytes(void) { return kStaticScratchBytes; }

extern "C" int ls_apply_noalloc(const dbi_model *model, const dbi_batch *batch, const void *Ghat,
                                const void *u, void *out, int precision, dbi_stream stream) {
  clear_error();
  int rc;
  if (!model) { set_error("model is NULL"); return DBI_ERR_ARG; }
  if ((rc = check_grid(&model->grid, precision)) || (rc = check_batch(batch)) || (rc = check_precision(precision))) return rc;
  const size_t need = dbi_workspace_bytes(&model->grid, batch->B, precision, DBI_OP_APPLY);
  if (need > kStaticScratchBytes) {
    set_error("ls_apply_noalloc: %d problems of %d x %d cells (FFT grid %d x %d) need %zu bytes of scratch, "
              "more than the fixed %zu bytes; split the batch or use ls_apply with a work buffer",
              batch->B, model->grid.nz, model->grid.nx, model->grid.lz, model->grid.lx, need,
              kStaticScratchBytes);
    return DBI_ERR_WORKSPACE;
  }
  if (batch->B == 0) return DBI_OK;
  void *scratch = nullptr;
  if ((rc = scratch_address(&scratch))) return rc;
  return ls_apply(model, batch, Ghat, u, out, precision, scratch, kStaticScratchBytes, stream);
}
