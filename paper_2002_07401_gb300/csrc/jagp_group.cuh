// jagp_group.cuh -- grouped launches: one launch of a kernel over the work of
// many independent systems (internal to libjagp).
//
// A kernel body is written as a functor F with
//   static __device__ void run(args..., uint3 bid, uint3 gdim)
// where bid / gdim stand for blockIdx / gridDim.  Its own __global__ kernel
// (the per-system launch) calls F::run(args..., blockIdx, gridDim).  While a
// GroupRecorder is installed on the calling thread, the launcher records (F,
// grid, block, shared memory, the argument values) instead of launching; the
// batch builder issues the records of all systems that sit at the same point
// of the sweep as ONE launch of k_run<F> (or k_run_global<F>): a 1-D grid that
// concatenates the systems' grids, in which a CTA finds its system (entry) by
// a binary search over the entries' first blocks (a kernel parameter, read
// through the constant cache) and runs F::run with that system's arguments
// and its block index within that system's grid.  Every CTA runs the same
// formulas in the same order as in the per-system launch; the compiled code
// differs (arguments read from memory instead of kernel parameters), so
// floating-point results may differ in the last bits where the compiler fused
// a multiply and an add differently.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <atomic>
#include <type_traits>
#include <utility>
#include <vector>

namespace jagp {

// a flat, trivially copyable pack of kernel arguments (the same layout on host and device)
template <class... A>
struct Pack;
template <>
struct Pack<> {};
template <class H, class... R>
struct Pack<H, R...> {
  H h;
  Pack<R...> r;
};

template <size_t I>
struct PGet {
  template <class P>
  __host__ __device__ __forceinline__ static const auto &get(const P &p) {
    return PGet<I - 1>::get(p.r);
  }
};
template <>
struct PGet<0> {
  template <class P>
  __host__ __device__ __forceinline__ static const auto &get(const P &p) {
    return p.h;
  }
};

inline void pack_fill(Pack<> &) {}
template <class H, class... R>
inline void pack_fill(Pack<H, R...> &p, const H &h, const R &...r) {
  p.h = h;
  pack_fill(p.r, r...);
}

template <class F, class P, size_t... I>
__device__ __forceinline__ void group_call(const P &p, uint3 bid, uint3 gd, std::index_sequence<I...>) {
  F::run(PGet<I>::get(p)..., bid, gd);
}

// The entries of one launch: entry e owns the flat blocks start[e] ..
// start[e + 1] - 1 and has the grid dims[e].
constexpr int kGroupMax = 64;
struct GroupTable {
  int n;
  int start[kGroupMax + 1];
  int dims[kGroupMax][3];
};

// minimum resident CTAs per SM that a functor asks of the compiler (F::kMinBlocks, default 1)
template <class F, class = void>
struct MinBlocks {
  static constexpr int value = 1;
};
template <class F>
struct MinBlocks<F, std::void_t<decltype(F::kMinBlocks)>> {
  static constexpr int value = F::kMinBlocks;
};

// The grouped launch of F: entries' arguments tab[e] in global memory, staged
// in shared memory so that the body reads them as cheaply as kernel parameters.
template <class F, int MT, class... A>
__global__ void __launch_bounds__(MT, MinBlocks<F>::value) k_run(const Pack<A...> *__restrict__ tab,
                                                                  const __grid_constant__ GroupTable t) {
  const int b = (int)blockIdx.x;
  int lo = 0, hi = t.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.start[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int gx = t.dims[lo][0], gy = t.dims[lo][1], gz = t.dims[lo][2];
  const int loc = b - t.start[lo];
  const uint3 bid = make_uint3((unsigned)(loc % gx), (unsigned)((loc / gx) % gy), (unsigned)(loc / (gx * gy)));
  const uint3 gd = make_uint3((unsigned)gx, (unsigned)gy, (unsigned)gz);
  using P = Pack<A...>;
  __shared__ __align__(16) uint32_t sp[(sizeof(P) + 3) / 4];
  const uint32_t *w = reinterpret_cast<const uint32_t *>(tab + lo);
  for (int i = (int)threadIdx.x; i < (int)(sizeof(P) / 4); i += (int)(blockDim.x * blockDim.y * blockDim.z))
    sp[i] = w[i];
  __syncthreads();
  group_call<F>(*reinterpret_cast<const P *>(sp), bid, gd, std::index_sequence_for<A...>{});
}

// The grouped launch of F with large or 64-byte aligned arguments (tensor
// maps, which must stay in global memory): read in place.
template <class F, int MT, class... A>
__global__ void __launch_bounds__(MT) k_run_global(const Pack<A...> *__restrict__ tab,
                                                    const __grid_constant__ GroupTable t) {
  const int b = (int)blockIdx.x;
  int lo = 0, hi = t.n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (t.start[mid] <= b)
      lo = mid;
    else
      hi = mid - 1;
  }
  const int gx = t.dims[lo][0], gy = t.dims[lo][1], gz = t.dims[lo][2];
  const int loc = b - t.start[lo];
  const uint3 bid = make_uint3((unsigned)(loc % gx), (unsigned)((loc / gx) % gy), (unsigned)(loc / (gx * gy)));
  group_call<F>(tab[lo], bid, make_uint3((unsigned)gx, (unsigned)gy, (unsigned)gz), std::index_sequence_for<A...>{});
}

// One recorded launch of one system.
struct GroupRecord {
  const void *fn = nullptr;  // the k_run / k_run_global instance (kernel and template arguments)
  dim3 grid, block;
  size_t smem = 0;
  std::vector<unsigned char> args;  // one Pack<A...>
  size_t align = 8;
  int key[5] = {0, 0, 0, 0, 0};  // the point of the sweep (set by group_key / group_subkey), then
  int seq = 0;                   // the launch's place at that point
  int sys = 0;
  int lane = 0;                  // chain of grouped launches it joins
};

// Collects the launches of one system's sweep (installed per thread by the
// batch builder; launchers consult group_recorder()).
struct GroupRecorder {
  int sys = 0;
  int key[5] = {0, 0, 0, 0, 0};
  int seq = 0;
  std::vector<GroupRecord> recs;
};

// the recorder installed on this thread (null: launch normally)
GroupRecorder *group_recorder();
void set_group_recorder(GroupRecorder *r);
// mark the point of the sweep that the following launches belong to
inline void group_key(int a, int b, int c, int d) {
  if (GroupRecorder *r = group_recorder()) {
    r->key[0] = a;
    r->key[1] = b;
    r->key[2] = c;
    r->key[3] = d;
    r->key[4] = 0;
    r->seq = 0;
  }
}
// a finer point within the current one (e.g. the steps of a refresh)
inline void group_subkey(int e) {
  if (GroupRecorder *r = group_recorder()) {
    r->key[4] = e;
    r->seq = 0;
  }
}

// allow kernel fn dynamic shared memory up to the current device's opt-in
// limit less its static shared memory; done[device] records that it was set
// (setting it twice from two threads is harmless)
cudaError_t group_raise_smem(const void *fn, std::atomic<unsigned char> *done);

// kernel<<<grid, block, smem, st>>>(a...) (the per-system launch of functor
// F, max. threads per block MT), or, while a recorder is installed, the
// record of that launch for a grouped launch of F.
template <class F, int MT, class K, class... A>
cudaError_t launch_or_record(K kernel, dim3 grid, dim3 block, size_t smem, cudaStream_t st, A... a) {
  if (GroupRecorder *R = group_recorder()) {
    const long long blocks = (long long)grid.x * grid.y * grid.z;
    if (blocks == 0) return cudaSuccess;
    if ((int)(block.x * block.y * block.z) > MT || blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    using P = Pack<A...>;
    P p{};
    pack_fill(p, a...);
    GroupRecord r;
    if constexpr (alignof(P) <= 16 && sizeof(P) <= 1024)
      r.fn = reinterpret_cast<const void *>(&k_run<F, MT, A...>);
    else
      r.fn = reinterpret_cast<const void *>(&k_run_global<F, MT, A...>);
    r.grid = grid;
    r.block = block;
    r.smem = smem;
    r.args.resize(sizeof(p));
    memcpy(r.args.data(), &p, sizeof(p));
    r.align = alignof(P);
    memcpy(r.key, R->key, sizeof(r.key));
    r.seq = R->seq++;
    r.sys = R->sys;
    R->recs.push_back(std::move(r));
    return cudaSuccess;
  }
  if (smem > 48 * 1024) {
    static std::atomic<unsigned char> raised[64];  // per device (zero at start)
    const cudaError_t e = group_raise_smem(reinterpret_cast<const void *>(kernel), raised);
    if (e != cudaSuccess) return e;
  }
  kernel<<<grid, block, smem, st>>>(a...);
  return cudaGetLastError();
}

// zero n ints at p on the stream (recorded as a grouped launch while recording)
cudaError_t zero_ints(int *p, int n, cudaStream_t st);

}  // namespace jagp
