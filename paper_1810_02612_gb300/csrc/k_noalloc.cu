// lbl_label_blocks_noalloc: the block-form labeling for callers that may not
// allocate device memory.
//
// The block-form kernel needs one piece of working memory besides its inputs
// and outputs: the bit-plane copy of the proposition words (one 64-bit word per
// 64-cell block and proposition).  lbl_label keeps it in the roadmap object,
// which lbl_roadmap_upload allocates.  Here it is a fixed, file-scope device
// array instead, so no call allocates or frees anything.  Everything else is
// the caller's memory, and the kernels are the ones lbl_label runs.
#include <mutex>

#include "lbl_internal.cuh"

namespace {

// The fixed working memory: 2^19 words = 4 MiB, held by every GPU that loads
// the library until the process exits.
constexpr int64_t kMaxPlaneWords = LBL_NOALLOC_MAX_PLANE_WORDS;
static __device__ __align__(256) uint64_t g_noalloc_planes[kMaxPlaneWords];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
uint64_t *g_planes_addr[kMaxDevices] = {nullptr};  // device address of g_noalloc_planes, per device
int g_num_sms[kMaxDevices] = {0};

// With the device current: in host code the array's name is only a stand-in,
// so ask the runtime for its device address.  The address is looked up again
// on every call whose stream is not being captured (a host application may
// have reset the device since, which reloads the module and can move the
// array); a call on a capturing stream reuses the address of the last lookup
// on this device, so the first call on a device, and the first after a
// cudaDeviceReset, must come before any capture.
int setup(int dev, bool lookup, uint64_t **planes, int *num_sms) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (lookup || !g_planes_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_planes);
    if (e != cudaSuccess) return lbl::cuda_fail(e, "label blocks (no alloc): cudaGetSymbolAddress");
    int n = 0;
    e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return lbl::cuda_fail(e, "label blocks (no alloc): SM count");
    g_num_sms[dev] = n > 0 ? n : 1;
    g_planes_addr[dev] = static_cast<uint64_t *>(p);
  }
  *planes = g_planes_addr[dev];
  *num_sms = g_num_sms[dev];
  return LBL_OK;
}

}  // namespace

extern "C" int lbl_label_blocks_noalloc(const int64_t *d_block_rowptr, const uint32_t *d_block_id,
                                        const uint64_t *d_block_mask, int64_t n_edges, const uint64_t *d_O,
                                        int64_t n_cells, int32_t n_props, uint64_t *d_L, lbl_stream s) {
  lbl::set_error("%s", "");
  if (n_edges < 0 || n_cells < 0 || n_cells > 2147483647LL || n_props < 0 || n_props > 64) {
    lbl::set_error("label blocks (no alloc): need n_edges >= 0, 0 <= n_cells < 2^31, 0 <= n_props <= 64");
    return LBL_EINVAL;
  }
  const int64_t n_blocks = (n_cells + 63) / 64;
  if (n_blocks > kMaxPlaneWords || n_blocks * n_props > kMaxPlaneWords) {
    lbl::set_error("label blocks (no alloc): %lld blocks x %d propositions need %lld plane words, more than the "
                   "fixed %lld (LBL_NOALLOC_MAX_PLANE_WORDS); use lbl_label instead",
                   static_cast<long long>(n_blocks), n_props, static_cast<long long>(n_blocks * n_props),
                   static_cast<long long>(kMaxPlaneWords));
    return LBL_EINVAL;
  }
  if (n_edges == 0) return LBL_OK;
  if (!d_block_rowptr || !d_L || (n_cells > 0 && n_props > 0 && !d_O)) {
    lbl::set_error("label blocks (no alloc): NULL buffer");
    return LBL_EINVAL;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return lbl::cuda_fail(e, "label blocks (no alloc): cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) {
    lbl::set_error("label blocks (no alloc): device %d beyond the %d supported", dev, kMaxDevices);
    return LBL_EUNSUPPORTED;
  }
  const cudaStream_t st = reinterpret_cast<cudaStream_t>(s);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) {
    (void)cudaGetLastError();  // e.g. the legacy stream while another stream captures: treat as capturing
    cap = cudaStreamCaptureStatusActive;
  }
  uint64_t *planes = nullptr;
  int num_sms = 1;
  int rc = setup(dev, cap == cudaStreamCaptureStatusNone, &planes, &num_sms);
  if (rc != LBL_OK) return rc;
  // A roadmap view over the caller's arrays: the same launch as lbl_label with
  // LBL_ALGO_BITTILE and its default (no early exit), with the fixed array as
  // its bit-plane memory.
  lbl::Roadmap view;
  view.device = dev;
  view.num_sms = num_sms;
  view.E = n_edges;
  view.cells = n_cells;
  view.has_bt = true;
  view.n_blocks = n_blocks;
  view.bt_rowptr = const_cast<int64_t *>(d_block_rowptr);
  view.bt_block = const_cast<uint32_t *>(d_block_id);
  view.bt_mask = const_cast<uint64_t *>(d_block_mask);
  view.planes = planes;
  e = lbl::launch_label_bittile(view, d_O, n_props, d_L, nullptr, false, 0, st);
  if (e != cudaSuccess) return lbl::cuda_fail(e, "label blocks (no alloc): launch");
  return LBL_OK;
}
