// Device helpers for the scan kernels (sm_103a).
//
//  * shared-memory staging windows filled by the Blackwell bulk-copy engine
//    (cp.async.bulk global -> shared, completion on an mbarrier), with every
//    wait bounded: a wait that runs out records DERR_TIMEOUT and the caller
//    returns instead of spinning;
//  * the device error word (first error wins, flags accumulate);
//  * ULEB128 varints and LSB-first bit extraction from staged bytes.
#pragma once
#include <stdint.h>

#include "pq_internal.h"

namespace pqi {

// Upper bound on mbarrier polls before a wait is declared lost.  Each poll
// may suspend in hardware for a while, so this is many seconds of waiting.
constexpr uint32_t kMaxPolls = 1u << 24;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void report(DevStatus* st, uint32_t flag, int page, int where, int detail) {
  atomicOr(&st->flags, flag);
  if (atomicCAS(&st->first_page, -1, page) == -1) {
    st->where = where;
    st->detail = detail;
  }
}

// ------------------------------------------------------------- mbarrier / TMA

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for phase `parity` of `bar`.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  for (uint32_t i = 0; i < kMaxPolls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// 1-D bulk copy global -> shared (dst, src 16-byte aligned, bytes % 16 == 0).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// A staging window: smem[0 .. n) holds global bytes [g0, g0 + n).  The smem
// buffer has `cap` + 16 bytes so that 8-byte reads just past n stay inside it.
struct Win {
  uint8_t* s;
  const uint8_t* g0;
  uint32_t cap;
  uint32_t n;
  uint64_t* bar;
  uint32_t parity;
};

// Block-collective: stage [from, min(limit, from + cap)) rounded out to 16
// bytes.  `limit` is the end of the stream; the rounding may read up to 15
// bytes on either side, which the engine guarantees to be readable (file
// buffers end with a footer, scratch buffers are padded).  Every thread
// must call it; returns false (after recording the timeout) if the copy
// never completed.
__device__ __forceinline__ bool win_load(Win& w, const uint8_t* from, const uint8_t* limit, DevStatus* st,
                                         int page, int where) {
  const uint8_t* a = reinterpret_cast<const uint8_t*>(reinterpret_cast<uintptr_t>(from) & ~uintptr_t(15));
  uint64_t want = static_cast<uint64_t>(limit - a);
  want = (want + 15) & ~uint64_t(15);
  uint32_t bytes = static_cast<uint32_t>(want < w.cap ? want : w.cap);
  if (bytes == 0) bytes = 16;
  __syncthreads();  // all generic reads of the previous contents are done
  if (threadIdx.x == 0) {
    fence_proxy_async_smem();
    mbar_arrive_expect_tx(w.bar, bytes);
    bulk_g2s(w.s, a, bytes, w.bar);
  }
  bool ok = mbar_wait(w.bar, w.parity);
  w.parity ^= 1u;
  w.g0 = a;
  w.n = bytes;
  if (!ok) {
    if (threadIdx.x == 0) report(st, DERR_TIMEOUT, page, where, 1);
    // wait (bounded) once more for the copy still in flight before the
    // shared buffer can be abandoned
    mbar_wait(w.bar, w.parity ^ 1u);
  }
  __syncthreads();
  return ok;
}

// ------------------------------------------------------------- byte readers

__device__ __forceinline__ uint32_t ld_u8(const uint8_t* p) { return __ldg(p); }

__device__ __forceinline__ uint32_t ld_le32_g(const uint8_t* p) {
  return ld_u8(p) | (ld_u8(p + 1) << 8) | (ld_u8(p + 2) << 16) | (ld_u8(p + 3) << 24);
}

// Reads a ULEB128 (<= 10 bytes) from bytes [p, end).  Returns the number of
// bytes consumed, 0 on overrun or overlong encoding.
template <typename Get>
__device__ __forceinline__ int uleb(Get get, uint32_t p, uint32_t end, uint64_t* v) {
  uint64_t r = 0;
  for (int i = 0; i < 10; ++i) {
    if (p + i >= end) return 0;
    uint32_t b = get(p + i);
    r |= static_cast<uint64_t>(b & 0x7f) << (7 * i);
    if (!(b & 0x80)) {
      *v = r;
      return i + 1;
    }
  }
  return 0;
}

__device__ __forceinline__ int64_t unzigzag(uint64_t u) {
  return static_cast<int64_t>(u >> 1) ^ -static_cast<int64_t>(u & 1);
}

// `w` 32-bit little-endian word view of a staged window; bit position `b`
// relative to the window's first byte.  Extracts `width` <= 32 bits.
__device__ __forceinline__ uint32_t bits32(const uint32_t* w, uint64_t b, int width) {
  uint32_t i = static_cast<uint32_t>(b >> 5);
  uint64_t pair = static_cast<uint64_t>(w[i]) | (static_cast<uint64_t>(w[i + 1]) << 32);
  uint64_t v = pair >> (b & 31);
  return width >= 32 ? static_cast<uint32_t>(v) : static_cast<uint32_t>(v & ((1ull << width) - 1));
}

// Same, `width` <= 64.
__device__ __forceinline__ uint64_t bits64(const uint32_t* w, uint64_t b, int width) {
  if (width <= 32) return bits32(w, b, width);
  uint32_t i = static_cast<uint32_t>(b >> 5);
  uint32_t s = static_cast<uint32_t>(b & 31);
  uint64_t lo = static_cast<uint64_t>(w[i]) | (static_cast<uint64_t>(w[i + 1]) << 32);
  uint64_t hi = w[i + 2];
  uint64_t v = s ? ((lo >> s) | (hi << (64 - s))) : lo;
  return width >= 64 ? v : (v & ((1ull << width) - 1));
}

// Unaligned little-endian load of 4 or 8 bytes from global memory, using
// aligned loads of the enclosing words (never reads outside the 8-byte
// aligned words that contain the value).
// Asks L2 to fetch the 128-byte lines of [p, end) (the warp's lanes take
// every 32nd line).  A hint only: nothing waits for it.  `end` must not pass
// the end of the buffer that holds p.
__device__ __forceinline__ void prefetch_l2(const uint8_t* p, const uint8_t* end, int lane) {
  const uintptr_t e = reinterpret_cast<uintptr_t>(end);
  for (uintptr_t a = (reinterpret_cast<uintptr_t>(p) & ~uintptr_t(127)) + 128u * lane; a < e; a += 32u * 128u)
    asm volatile("prefetch.global.L2 [%0];" ::"l"(a));
}

__device__ __forceinline__ uint64_t ld_unaligned_g(const uint8_t* p, int width) {
  uintptr_t a = reinterpret_cast<uintptr_t>(p);
  const uint64_t* q = reinterpret_cast<const uint64_t*>(a & ~uintptr_t(7));
  uint32_t s = static_cast<uint32_t>(a & 7) * 8;
  uint64_t lo = __ldg(q);
  if (s == 0) return width == 8 ? lo : (lo & 0xffffffffull);
  uint64_t v = lo >> s;
  if (s + 8u * width > 64) v |= __ldg(q + 1) << (64 - s);
  return width == 8 ? v : (v & 0xffffffffull);
}

// Block-wide exclusive sum over one value per thread (blockDim.x <= 1024,
// multiple of 32).  `tmp` needs 32 entries.  Returns the thread's prefix;
// *total receives the block total.
template <typename T>
__device__ __forceinline__ T block_exclusive_sum(T v, T* tmp, T* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  T x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  __syncthreads();
  if (lane == 31) tmp[warp] = x;
  __syncthreads();
  if (warp == 0) {
    T t = lane < nw ? tmp[lane] : T(0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    if (lane < nw) tmp[lane] = t;
  }
  __syncthreads();
  T before = warp ? tmp[warp - 1] : T(0);
  *total = tmp[nw - 1];
  __syncthreads();
  return before + x - v;
}


// ------------------------------------------------------------- warp copies

template <bool kReadOnly, typename T>
__device__ __forceinline__ T ld_src(const T* p) {
  if constexpr (kReadOnly) return __ldg(p);
  else return *reinterpret_cast<const volatile T*>(p);
}
template <>
__device__ __forceinline__ uint4 ld_src<false, uint4>(const uint4* p) {
  uint4 v;
  asm volatile("ld.global.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p) : "memory");
  return v;
}
template <>
__device__ __forceinline__ uint8_t ld_src<false, uint8_t>(const uint8_t* p) {
  uint16_t v;
  asm volatile("ld.global.u8 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
  return static_cast<uint8_t>(v);
}

// 16 bytes starting at byte s (0..15) of the 32-byte pair (A, B); the word
// offset s >> 2 is warp-uniform, so the switch does not diverge.
__device__ __forceinline__ uint4 shift_pair(const uint4& A, const uint4& B, uint32_t s) {
  const uint32_t bs = (s & 3) * 8;
  uint32_t w0, w1, w2, w3, w4;
  switch (s >> 2) {
    case 0: w0 = A.x; w1 = A.y; w2 = A.z; w3 = A.w; w4 = B.x; break;
    case 1: w0 = A.y; w1 = A.z; w2 = A.w; w3 = B.x; w4 = B.y; break;
    case 2: w0 = A.z; w1 = A.w; w2 = B.x; w3 = B.y; w4 = B.z; break;
    default: w0 = A.w; w1 = B.x; w2 = B.y; w3 = B.z; w4 = B.w; break;
  }
  return make_uint4(__funnelshift_r(w0, w1, bs), __funnelshift_r(w1, w2, bs), __funnelshift_r(w2, w3, bs),
                    __funnelshift_r(w3, w4, bs));
}

// One warp copies `bytes` bytes from `src` (any alignment) to `dst` (aligned
// to the value width): bytes up to dst's 16-byte boundary one by one, then
// 16-byte stores built from aligned 16-byte loads (8 per lane in flight; the
// next aligned word comes from the neighbouring lane by a shuffle), then the
// tail.  Reads may reach 16 bytes past src + bytes.  kReadOnly: the source
// is not written by the running kernel (non-coherent loads); otherwise the
// loads are coherent (a copy out of the kernel's own output).
__device__ __forceinline__ uint4 shfl_u4(const uint4& v, int src_lane) {
  return make_uint4(__shfl_sync(0xffffffffu, v.x, src_lane), __shfl_sync(0xffffffffu, v.y, src_lane),
                    __shfl_sync(0xffffffffu, v.z, src_lane), __shfl_sync(0xffffffffu, v.w, src_lane));
}
__device__ __forceinline__ uint4 shfl_down_u4(const uint4& v) {
  return make_uint4(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1),
                    __shfl_down_sync(0xffffffffu, v.z, 1), __shfl_down_sync(0xffffffffu, v.w, 1));
}

template <bool kReadOnly = true>
__device__ __forceinline__ void warp_copy(uint8_t* dst, const uint8_t* src, uint64_t bytes, int lane) {
  const uint32_t head0 = static_cast<uint32_t>((16 - (reinterpret_cast<uintptr_t>(dst) & 15)) & 15);
  const uint32_t head = head0 < bytes ? head0 : static_cast<uint32_t>(bytes);
  if (static_cast<uint32_t>(lane) < head) dst[lane] = ld_src<kReadOnly>(src + lane);
  dst += head;
  src += head;
  bytes -= head;
  const uint64_t nvec = bytes >> 4;
  const uint32_t s = static_cast<uint32_t>(reinterpret_cast<uintptr_t>(src) & 15);
  const uint4* sa = reinterpret_cast<const uint4*>(src - s);
  uint4* dv = reinterpret_cast<uint4*>(dst);
  constexpr int U = 8;
  for (uint64_t v0 = 0; v0 < nvec; v0 += 32 * U) {
    uint4 A[U];
    uint4 X = make_uint4(0, 0, 0, 0);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = v0 + u * 32 + lane;
      A[u] = i <= nvec ? ld_src<kReadOnly>(sa + i) : make_uint4(0, 0, 0, 0);
    }
    if (s && lane == 0 && v0 + 32 * U <= nvec) X = ld_src<kReadOnly>(sa + v0 + 32 * U);
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const uint64_t i = v0 + u * 32 + lane;
      uint4 out = A[u];
      if (s) {  // warp-uniform
        const uint4 dn = shfl_down_u4(A[u]);
        const uint4 nx = shfl_u4(u + 1 < U ? A[u + 1] : X, 0);
        out = shift_pair(A[u], lane == 31 ? nx : dn, s);
      }
      if (i < nvec) dv[i] = out;
    }
  }
  const uint32_t tail = static_cast<uint32_t>(bytes & 15);
  if (static_cast<uint32_t>(lane) < tail) dst[(nvec << 4) + lane] = ld_src<kReadOnly>(src + (nvec << 4) + lane);
}


}  // namespace pqi
