// Tensor-memory-accelerator (TMA) tile copies between global memory and
// shared memory, completed on an mbarrier (loads) or a bulk group (stores),
// and the host-side encoding of the tensor maps they read.
#pragma once
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstring>
#include <map>
#include <mutex>
#include <tuple>

namespace rvk {

// ------------------------------------------------------------------ device
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Count `bytes` as arrived on the barrier's transaction counter without a
// copy (used when a CTA gives up on a tile whose expected count exceeds what
// its copy delivers, so that the phase still completes once the copy lands).
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.complete_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Wait for phase `parity` of the barrier for at most max_ns nanoseconds;
// false when that budget ran out.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, unsigned long long max_ns) {
  const uint32_t a = smem_u32(bar);
  const unsigned long long t0 = global_ns();
  for (;;) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > max_ns) return false;
  }
}

// 4D tile load of the tensor map's box at (c0, c1, c2, c3) into dst; the
// bytes are counted on bar.
__device__ __forceinline__ void tma_load_4d(void* dst, const CUtensorMap* map, int c0, int c1, int c2, int c3,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_u32(bar))
      : "memory");
}

// 4D tile store of src to the tensor map's box at (c0, c1, c2, c3), then
// wait until the source has been read (the shared memory may be released).
// The writes to src must be made visible to the async proxy first
// (tma_fence_smem by every writing thread, then a barrier).
__device__ __forceinline__ void tma_store_4d_and_wait(const CUtensorMap* map, const void* src, int c0, int c1,
                                                      int c2, int c3) {
  asm volatile(
      "cp.async.bulk.tensor.4d.global.shared::cta.tile.bulk_group [%0, {%2, %3, %4, %5}], [%1];" ::"l"(
          reinterpret_cast<uint64_t>(map)),
      "r"(smem_u32(src)), "r"(c0), "r"(c1), "r"(c2), "r"(c3)
      : "memory");
  asm volatile("cp.async.bulk.commit_group;" ::: "memory");
  asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory");
}

__device__ __forceinline__ void tma_fence_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// ------------------------------------------------------------------ host
// Tiled tensor map over 8-byte elements: dims[0] innermost (contiguous),
// strides in bytes for dims 1..rank-1.  Maps are cached by their
// parameters (encoding is a driver call); nullptr when the driver entry
// point or the encoding is not available.
using TmapKey = std::tuple<void*, int, unsigned long long, unsigned long long, unsigned long long,
                           unsigned long long, unsigned long long, unsigned long long, unsigned long long,
                           unsigned, unsigned, unsigned, unsigned>;

struct TmapCache {
  std::mutex mu;
  std::map<TmapKey, CUtensorMap*> maps;
  PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  bool tried = false;
};

// one cache for the whole library (an inline function's static is unique)
inline TmapCache& tmap_cache() {
  static TmapCache c;
  return c;
}

// Drop the cached maps over a buffer that is about to be freed (a later
// allocation at the same address must get maps of its own shapes).
inline void tensor_map_evict_impl(const void* base) {
  TmapCache& c = tmap_cache();
  std::lock_guard<std::mutex> lock(c.mu);
  for (auto it = c.maps.begin(); it != c.maps.end();) {
    if (std::get<0>(it->first) == base) {
      delete it->second;
      it = c.maps.erase(it);
    } else {
      ++it;
    }
  }
}

inline const CUtensorMap* tensor_map_8b(void* base, int rank, const unsigned long long* dims,
                                        const unsigned long long* strides, const unsigned* box) {
  using Key = TmapKey;
  TmapCache& c = tmap_cache();
  std::mutex& mu = c.mu;
  std::map<Key, CUtensorMap*>& cache = c.maps;
  PFN_cuTensorMapEncodeTiled_v12000& encode = c.encode;
  bool& tried = c.tried;
  unsigned long long d[4] = {1, 1, 1, 1}, s[3] = {0, 0, 0};
  unsigned b[4] = {1, 1, 1, 1};
  for (int i = 0; i < rank; i++) { d[i] = dims[i]; b[i] = box[i]; }
  for (int i = 0; i + 1 < rank; i++) s[i] = strides[i];
  const Key key{base, rank, d[0], d[1], d[2], d[3], s[0], s[1], s[2], b[0], b[1], b[2], b[3]};
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  if (!tried) {
    tried = true;
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    else
      cudaGetLastError();
  }
  if (!encode) return nullptr;
  cuuint64_t gd[4];
  cuuint64_t gs[3];
  cuuint32_t bx[4], es[4] = {1, 1, 1, 1};
  for (int i = 0; i < rank; i++) { gd[i] = d[i]; bx[i] = b[i]; }
  for (int i = 0; i + 1 < rank; i++) gs[i] = s[i];
  CUtensorMap* m = new CUtensorMap;
  std::memset(m, 0, sizeof(*m));
  const CUresult r = encode(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, (cuuint32_t)rank, base, gd, gs, bx, es,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    delete m;
    m = nullptr;
  }
  cache[key] = m;
  return m;
}

}  // namespace rvk
