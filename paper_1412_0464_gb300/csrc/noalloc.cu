// hz_slab_solve_noalloc: a slab solve that allocates no device memory.
//
// Some callers must not allocate device memory once they are running:
// real-time or embedded schedulers that forbid allocation after
// initialisation, and applications that hand the whole device memory to their
// own pool allocator (a cudaMalloc inside the library could then fail, or
// fragment the pool).  This entry point serves them: its work buffers live in
// one fixed device array defined below, so the call itself never allocates.
//
// The array is a file-scope __device__ variable: every GPU that loads this
// library holds kScratchBytes of it until the process exits.  In host code
// the name g_slab_scratch is only a host-side stand-in for the symbol, not a
// device address; passing it to a kernel would fault (or, where the GPU can
// reach host memory, silently use the wrong memory).  The device address is
// obtained once per device with cudaGetSymbolAddress, with that device
// current, on the first call made on that device, and kept for the life of
// the process (calls after cudaDeviceReset are not supported).
#include "hz_internal.h"

#include <mutex>

namespace {

constexpr size_t kScratchBytes = 8u << 20;   // 8 MiB
constexpr int kMaxDevices = 128;

static __device__ __align__(256) unsigned char g_slab_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of g_slab_scratch on the current device (looked up once).
void* scratch_address() {
  int dev = 0;
  HZ_CU(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw hz::Failure(HZ_EINVAL, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_slab_scratch);
    if (e != cudaSuccess || !p)
      throw hz::Failure(HZ_ECUDA, std::string("cudaGetSymbolAddress(slab scratch) failed: ") +
                                      cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

using namespace hz;

extern "C" hz_status hz_slab_solve_noalloc(hz_handle* h, int j, const hz_c128* f_dev,
                                           hz_c128* u_dev, int n_rhs, void* stream) {
  if (!h) return HZ_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  return run_guarded(h, [&] {
    if (!h->sweep) throw Failure(HZ_EINVAL, "handle has no sweep level");
    Level& L = *h->sweep;
    if (j < 1 || j > L.J) throw Failure(HZ_EINVAL, "slab index out of range");
    if (n_rhs < 1 || n_rhs > h->p.max_rhs) throw Failure(HZ_EINVAL, "n_rhs out of range");
    if (!f_dev || !u_dev) throw Failure(HZ_EINVAL, "NULL field pointer");
    if (L.dim3d) throw Failure(HZ_EINVAL, "the no-allocation slab solve serves 2-D slabs only");
    int dev = 0;
    HZ_CU(cudaGetDevice(&dev));
    if (dev != h->dev) throw Failure(HZ_EINVAL, "the handle's device is not the current device");
    const bool mixed = h->p.precision == HZ_MIXED;
    const size_t el = mixed ? sizeof(c64) : sizeof(c128);
    const size_t W = L.slabs[j].W, wp = L.slabs[j].wp;
    const size_t field = (size_t)n_rhs * L.ny * W;           // one slab-sized field
    const size_t rows = (size_t)n_rhs * L.ny * wp;           // forward rows (padded)
    const size_t carry_f = (size_t)(L.P + L.NG) * n_rhs * wp;       // forward carries, group ends
    const size_t carry_b = (size_t)(L.P + 1 + L.NG) * n_rhs * wp;   // backward ones, meeting row
    const size_t need = (mixed ? 2 * align256(field * el) : 0) + align256(rows * el) +
                        align256(carry_f * el) + align256(carry_b * el);
    if (need > kScratchBytes)
      throw Failure(HZ_EINVAL, "slab solve needs " + std::to_string(need) +
                                   " bytes of work space; the no-allocation entry point holds " +
                                   std::to_string(kScratchBytes) + " bytes");
    if (!h->factored) throw Failure(HZ_ENOTFACTORED, "hz_slab_solve_noalloc before hz_factor");
    unsigned char* base = (unsigned char*)scratch_address();
    // Every region below is written in full before it is read (right-hand
    // side copy, forward rows, segment carries), so nothing needs clearing.
    size_t off = 0;
    auto take = [&](size_t bytes) { void* p = base + off; off += align256(bytes); return p; };
    if (mixed) {
      c64* fd = (c64*)take(field * el);
      c64* ud = (c64*)take(field * el);
      c64* Y = (c64*)take(rows * el);
      c64* cf = (c64*)take(carry_f * el);
      c64* cb = (c64*)take(carry_b * el);
      cast_copy<float, double>((const c128*)f_dev, fd, field, s);
      slab_solve_raw_scratch<float>(h, L, j, fd, ud, n_rhs, s, Y, cf, cb);
      cast_copy<double, float>(ud, (c128*)u_dev, field, s);
    } else {
      c128* Y = (c128*)take(rows * el);
      c128* cf = (c128*)take(carry_f * el);
      c128* cb = (c128*)take(carry_b * el);
      slab_solve_raw_scratch<double>(h, L, j, (const c128*)f_dev, (c128*)u_dev, n_rhs, s, Y, cf,
                                     cb);
    }
    HZ_CU(cudaStreamSynchronize(s));
    check_dev_flag(h, s);
  });
}
