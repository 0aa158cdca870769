// Forward rasteriser that allocates nothing (tgs_raster_forward_noalloc).
//
// Some callers cannot allocate device memory at the point where they render:
// renderers that run inside a fixed, pre-reserved memory budget owned by
// another framework's allocator (a cudaMalloc of their own would fail or
// fragment that budget), or real-time loops that must not pay for an
// allocation or risk one failing mid-frame.  For them this entry point keeps every
// intermediate of the forward (per-Gaussian splats, visibility compaction,
// the depth and tile radix sorts, the pair lists, tile ranges and per-pixel
// state) in one file-scope device array of fixed size, g_noalloc_scratch.
//
// The array lives in every GPU that loads the library until the process
// exits.  Host code must not hand the symbol itself to a kernel: on the host
// the name is only a stand-in for the device object.  The first call on each
// device resolves the array's device address with cudaGetSymbolAddress (with
// that device current) and caches it; make that first call before any stream
// capture begins.  The call reads the visible and pair counts back to the host
// (it waits on `stream` twice) and returns after its work has completed.  All
// calls share the one array, which keeps the previous
// call's contents: what must start at zero (the tile ranges) is cleared by
// each call, and two calls whose GPU work overlaps (different streams, or
// different host threads) race on the array.
#include <mutex>

#include "raster.cuh"
#include "sort.cuh"

namespace tgs {
namespace {

constexpr size_t NOALLOC_BYTES = 16u << 20;       // 16 MiB
constexpr uint64_t NA_MAX_GAUSS = 32768;          // render-list positions (n rounded up to whole blocks)
constexpr uint64_t NA_MAX_PAIRS = 524288;         // (tile, Gaussian) pairs
constexpr uint64_t NA_MAX_PIX = 512ull * 512ull;  // image pixels
constexpr uint64_t NA_MAX_TILES = 1024;           // 16 x 16 tiles

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_mu;
void* g_base[MAX_DEVICES] = {nullptr};
// render-list staging (item slot / count / block); copied into the array
uint32_t g_rl_host[3 * NA_MAX_GAUSS];

struct Carver {
  unsigned char* base;
  size_t off = 0;
  template <class T>
  T* take(uint64_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = reinterpret_cast<T*>(base + off);
    off += count * sizeof(T);
    return p;
  }
};

void* device_base() {
  int dev = 0;
  TGS_CUDA(cudaGetDevice(&dev));
  TGS_CHECK(dev >= 0 && dev < MAX_DEVICES, TGS_ERR_INVALID, "device ordinal out of range");
  if (!g_base[dev]) {
    void* p = nullptr;
    TGS_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_base[dev] = p;
  }
  return g_base[dev];
}

}  // namespace
}  // namespace tgs

using namespace tgs;

extern "C" tgs_status tgs_raster_forward_noalloc(const float* params_dev, uint64_t n, uint32_t block_size,
                                                 const tgs_camera* cam, const float* bg3, float* image_dev,
                                                 void* stream) {
  try {
    set_last_error("");
    TGS_CHECK(params_dev && cam && image_dev, TGS_ERR_INVALID, "tgs_raster_forward_noalloc: null argument");
    TGS_CHECK(n >= 1 && block_size >= 1, TGS_ERR_INVALID, "tgs_raster_forward_noalloc: empty input");
    const uint64_t items = (n + block_size - 1) / block_size;
    TGS_CHECK(items * block_size <= NA_MAX_GAUSS, TGS_ERR_CAPACITY,
              "tgs_raster_forward_noalloc: ceil(n / block_size) * block_size exceeds 32768");
    DevCam dc = make_devcam(*cam);
    TGS_CHECK((uint64_t)dc.W * dc.H <= NA_MAX_PIX && (uint64_t)dc.TX * dc.TY <= NA_MAX_TILES, TGS_ERR_CAPACITY,
              "tgs_raster_forward_noalloc: image larger than 512 x 512 pixels");
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_mu);
    Carver cv{(unsigned char*)device_base()};
    const uint64_t V = NA_MAX_GAUSS, P = NA_MAX_PAIRS;
    CamState cs;
    cs.cap_v = V;
    cs.cap_pairs = P;
    cs.cap_pix = NA_MAX_PIX;
    cs.cap_tiles = NA_MAX_TILES;
    cs.xy = cv.take<float2>(V);
    cs.depth = cv.take<float>(V);
    cs.conic_o = cv.take<float4>(V);
    cs.rgb = cv.take<float4>(V);
    cs.rect = cv.take<ushort4>(V);
    cs.radius = cv.take<int>(V);
    cs.ntiles = cv.take<uint32_t>(V);
    cs.scan = cv.take<uint32_t>(V);
    cs.dkeys = cv.take<uint32_t>(2 * V);
    cs.dvals = cv.take<uint32_t>(2 * V);
    cs.pkeys = cv.take<uint32_t>(2 * P);
    cs.pvals = cv.take<uint32_t>(2 * P);
    cs.ranges = cv.take<uint2>(NA_MAX_TILES);
    cs.t_final = cv.take<float>(NA_MAX_PIX);
    cs.n_last = cv.take<int>(NA_MAX_PIX);
    cs.counters = cv.take<uint32_t>(4);
    uint32_t* rl_dev = cv.take<uint32_t>(3 * NA_MAX_GAUSS);
    size_t sb = radix_scratch_bytes(P);
    if (scan_scratch_bytes(P) > sb) sb = scan_scratch_bytes(P);
    cs.scratch = cv.take<unsigned char>(sb);
    cs.scratch_bytes = sb;
    TGS_CHECK(cv.off <= NOALLOC_BYTES, TGS_ERR_STATE, "no-alloc layout exceeds its static array");
    for (uint64_t j = 0; j < items; ++j) {
      g_rl_host[j] = (uint32_t)j;
      g_rl_host[items + j] = (uint32_t)std::min<uint64_t>(block_size, n - j * block_size);
      g_rl_host[2 * items + j] = (uint32_t)j;
    }
    TGS_CUDA(cudaMemcpyAsync(rl_dev, g_rl_host, 3 * items * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    RenderList rl;
    rl.base = const_cast<float*>(params_dev);
    rl.slot_stride = (uint64_t)D * block_size;
    rl.B = block_size;
    rl.n_items = (uint32_t)items;
    rl.item_slot = rl_dev;
    rl.item_count = rl_dev + items;
    rl.item_block = rl_dev + 2 * items;
    rl.m_off = rl.v_off = 0;
    float bg[3] = {0.f, 0.f, 0.f};
    if (bg3) {
      bg[0] = bg3[0];
      bg[1] = bg3[1];
      bg[2] = bg3[2];
    }
    render_forward_fixed(rl, dc, bg, cs, image_dev, s);
    // the pageable staging buffer must not be rewritten before its copy is done
    TGS_CUDA(cudaStreamSynchronize(s));
    return TGS_OK;
  } catch (const Error& e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    set_last_error(e.what());
    return TGS_ERR_INVALID;
  }
}
