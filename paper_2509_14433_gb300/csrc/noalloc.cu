// Sketch update for callers that cannot allocate device memory.
//
// cupc_update_sketch_static applies a batch of edge updates to a sketch
// buffer the caller owns, using the same kernels as cupc_update_batch. Its
// scratch (per-vertex counts and cursors, endpoint records, work items, hash
// keys, counters) is the file-scope array below instead of a workspace, so
// the call allocates nothing. The paper has no counterpart of this entry
// point.
#include <mutex>

#include "common.cuh"

using namespace cupc;

namespace {

constexpr uint32_t kMaxV = CUPC_STATIC_MAX_V;
constexpr uint32_t kMaxEdges = CUPC_STATIC_MAX_EDGES;
// key words of the widest graph: V = kMaxV has L = 18 layers, C = 7 columns
constexpr uint32_t kMaxKeys = (uint32_t)key_words(18, 7);
constexpr size_t kAlignS = 256;
constexpr size_t align_s(size_t x) { return (x + kAlignS - 1) / kAlignS * kAlignS; }
constexpr size_t kMaxItems =
    4ull * kMaxEdges / kMinItemRecords + (kMaxV < 2ull * kMaxEdges ? kMaxV : 2ull * kMaxEdges) + 2ull * kPlanGridCap + 1;
// byte offsets inside the static scratch
constexpr size_t kOffGc = 0;
constexpr size_t kOffKeys = align_s(kOffGc + GC_SLOTS * sizeof(uint32_t));
constexpr size_t kOffCnt = align_s(kOffKeys + kMaxKeys * sizeof(uint64_t));
constexpr size_t kOffCursor = align_s(kOffCnt + kMaxV * sizeof(uint32_t));
constexpr size_t kOffRec = align_s(kOffCursor + kMaxV * sizeof(uint32_t));
constexpr size_t kOffRecw = align_s(kOffRec + 2ull * kMaxEdges * sizeof(uint64_t));
constexpr size_t kOffItems = align_s(kOffRecw + 2ull * kMaxEdges * sizeof(uint32_t));
constexpr size_t kOffPart = align_s(kOffItems + kMaxItems * sizeof(uint4));
constexpr size_t kScratchBytes = align_s(kOffPart + kPlanSlices * sizeof(uint4));
static_assert(kScratchBytes == CUPC_STATIC_SCRATCH_BYTES, "the header states the size of the static scratch");

// Shared by every call on a device, kept between calls.
static __device__ __align__(256) unsigned char cupc_static_scratch[kScratchBytes];

// Per-device set-up: the device address of the scratch (the host-side name
// of the array is only a stand-in) and the launch shape of the apply kernel.
struct DeviceSetup {
  bool done;
  cudaError_t err;
  unsigned char* scratch;
  int sms, apply_threads, apply_smem, apply_grid;
  uint32_t P, R;
};
constexpr int kMaxDevices = 64;
DeviceSetup g_setup[kMaxDevices];
std::mutex g_setup_mutex;

uint32_t ceil_log2_s(uint32_t V) {
  uint32_t lg = 0;
  while (((uint64_t)1 << lg) < (uint64_t)V) lg++;
  return lg < 1 ? 1 : lg;
}

void fill_dims(cupc_graph& g, uint32_t V) {
  const uint32_t lg = ceil_log2_s(V);
  g.V = V;
  g.L = lg + 2;
  g.C = 7;
  g.D = 2 * lg;
  g.W = 1 + g.C * g.D;
}

// A set-up that fails is not kept: the next call on that device tries
// again (a failure can be transient, or the first call may have come during
// a stream capture).
cudaError_t device_setup(int dev, DeviceSetup** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& s = g_setup[dev];
  if (!s.done) {
    cudaError_t err = cudaGetSymbolAddress((void**)&s.scratch, cupc_static_scratch);
    if (err == cudaSuccess) err = cudaDeviceGetAttribute(&s.sms, cudaDevAttrMultiProcessorCount, dev);
    if (err == cudaSuccess) {
      // the widest apply launch: V = kMaxV sets the most layers
      cupc_graph g{};
      fill_dims(g, kMaxV);
      g.sms = s.sms;
      err = setup_update(&g);
      s.apply_threads = g.apply_threads;
      s.apply_smem = g.apply_smem;
      s.apply_grid = g.apply_grid;
      s.P = g.P;
      s.R = g.R;
    }
    if (err != cudaSuccess) {
      cudaGetLastError();  // clear it, so that a later call starts clean
      return err;
    }
    s.done = true;
  }
  *out = &s;
  return cudaSuccess;
}

// Device or managed memory (cudaPointerGetAttributes allocates nothing).
bool device_memory(const void* p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

extern "C" cupc_status cupc_update_sketch_static(void* sketch, uint32_t V, uint64_t seed, const uint32_t* edges,
                                                 const int8_t* ops, size_t n, uint32_t* status_out,
                                                 cupc_stream stream) {
  if (!sketch || V < 2 || V > kMaxV || n > kMaxEdges) return CUPC_EINVAL;
  if (n > 0 && (!edges || !ops)) return CUPC_EINVAL;
  // the kernels read and write these directly: a host address here would
  // fault on the GPU, so it is refused before any launch; the apply kernel
  // accesses the sketch 16 bytes at a time
  if (((uintptr_t)sketch & 15) != 0 || !device_memory(sketch)) return CUPC_EINVAL;
  if (n > 0 && (!device_memory(edges) || !device_memory(ops))) return CUPC_EINVAL;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CUPC_ECUDA;
  DeviceSetup* ds = nullptr;
  if (device_setup(dev, &ds) != cudaSuccess) return CUPC_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;

  cupc_graph g{};
  fill_dims(g, V);
  g.seed = seed;
  g.max_batch = kMaxEdges;
  g.sms = ds->sms;
  g.P = ds->P;
  g.R = g.D < kSmemRows ? g.D : kSmemRows;
  g.ell = hash_bits(V);
  g.long_depth = g.ell < g.D - 1 || g.D - 1 > 32;
  g.item_records = kDefaultItemRecords;
  g.apply_threads = (int)(((g.L * g.P) + 31) / 32 * 32);
  g.apply_smem = (int)apply_smem_bytes(g.R, (uint32_t)g.apply_threads, g.L);
  // the set-up sized the launch for the widest graph; a narrower one fits
  g.apply_grid = ds->apply_grid;
  g.prof_on = false;
  g.sketch = (ulonglong2*)sketch;
  g.gc = (uint32_t*)(ds->scratch + kOffGc);
  g.keys = (uint64_t*)(ds->scratch + kOffKeys);
  g.cnt = (uint32_t*)(ds->scratch + kOffCnt);
  g.cursor = (uint32_t*)(ds->scratch + kOffCursor);
  g.rec = (uint64_t*)(ds->scratch + kOffRec);
  g.recw = (uint32_t*)(ds->scratch + kOffRecw);
  g.items = (uint4*)(ds->scratch + kOffItems);
  g.part = (uint4*)(ds->scratch + kOffPart);

  // the array keeps the previous call's contents: clear what must start at 0
  if (cudaMemsetAsync(g.gc, 0, GC_SLOTS * sizeof(uint32_t), s) != cudaSuccess) return CUPC_ECUDA;
  if (cudaMemsetAsync(g.cnt, 0, (size_t)V * sizeof(uint32_t), s) != cudaSuccess) return CUPC_ECUDA;
  if (launch_keys(&g, s) != cudaSuccess) return CUPC_ECUDA;
  if (n > 0) {
    if (launch_validate(&g, edges, ops, n, s) != cudaSuccess) return CUPC_ECUDA;
    if (launch_update_chunk(&g, edges, n, s) != cudaSuccess) return CUPC_ECUDA;
  }
  if (status_out && cudaMemcpyAsync(status_out, g.gc + GC_ERR, sizeof(uint32_t), cudaMemcpyDefault, s) != cudaSuccess)
    return CUPC_ECUDA;
  return CUPC_OK;
}
