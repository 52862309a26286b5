// bm_step.cuh -- the fused step kernel (sm_103a): persistent CTAs of eight compute
// warps and one copy warp, a shared-memory pipeline fed by bulk asynchronous copies.
//
// CTAs take work items (tiles of 256 Hilbert-ordered cells of some instance) by
// ticket: a share of each CTA's tickets is static (known ahead, no atomic), the rest
// come from a launch-wide counter, so a CTA that meets expensive wet tiles simply takes
// fewer.  A launch takes the fixed items (tiles with boundary edges that carry mass,
// inflow, source or outflow tiles, and item 0) and then the items the previous launch
// listed: a tile that was not quiet lists itself and the tiles its halo cells lie in.
// Every other tile was quiet or skipped in the previous launch and has no changed
// neighbour: it is dry and at rest, both state buffers hold its values, and its step
// would copy them through, so the launch skips it (no copy, no record, no arithmetic).
// Where that is not allowed (passive species or bed evolution, whose kernels read
// every tile), and in the first launch after the state or its features changed (a
// "full" launch), every tile is taken: FP64 first the tiles the previous launch
// listed -- wet tiles cost many times a dry one at B300's FP64 rate and must not come
// last -- then the rest in the work list's (Hilbert) order, which FP32-bulk, bound by
// memory traffic, takes from the start.  Each tile's arithmetic and every reduction are
// order-independent or in a fixed order, so the result does not depend on which CTA
// took which tile, or when, or on which tiles were skipped.  Its copy warp streams every tile's data
// into a shared-memory slot ahead of the compute warps, in two groups completed on
// mbarriers:
//   group A  bulk copies (cp.async.bulk) of the tile record (inverse areas, slots,
//            edge codes and geometry, halo list), the instance descriptor, a snapshot
//            of its control block and the tile's slices of the state arrays (surface,
//            discharge, bed, g n^2) -- addresses the copy warp knows without waiting
//            (instance pointers cached per instance);
//   group H  issued right after A: cp.async gathers of the halo cells' values (other
//            tiles' cells, in ascending index order), the halo list read from the
//            record in global memory one tile ahead, so H does not wait for A.
// Three slots per CTA.  The compute warps release a slot when they are done with its
// tile; the copy warp polls for released slots and refills them, so copies run a few
// tiles ahead of the arithmetic.  The compute warps read shared memory only (BASEMENT v3,
// Section "Numerical solution"):
//   phase D  wet/dry flag, velocity and celerity of every local cell (dry: zero, without
//            arithmetic);
//            a tile whose cells and halo are dry, at rest and without inflow is quiet;
//   phase F  each tile edge once: modified states on max(z_L, z_R), HLLC flux in the
//            edge frame, pre-balanced pressure, wall / transmissive / inflow states;
//            an edge whose two cells are dry, or whose modified depths are both zero,
//            contributes exactly zero and is not evaluated;
//   phase I  each cell gathers its three edge contributions (Eq. 12), split Manning
//            friction (Eq. 2, Table 1), U^{n+1} to HBM, the lambda/rho rate of Eq. 21;
//            a dry cell at rest with three skipped edges (every cell of a quiet tile)
//            is copied through unchanged;
//   flush    when the CTA leaves an instance: its max rate to the instance's control
//            block; boundary volume and inflow split by the CTA that completes the
//            instance's last boundary / inflow tile; the next launch's lists;
//   end      the CTA that completes the launch finalizes every instance that stepped
//            (next dt, time, parity) and rolls the lists over -- no second launch.
// Every wait is bounded (about a second): on timeout the CTA flags the instance
// (status bit 2), its copy warp drains what it issued, and all warps return.
#pragma once

#include "bm_kernels.cuh"

namespace bm {

constexpr long long kWaitCycles = 2000000000LL;
constexpr int kStepThreads = kTile + 32;  // eight compute warps + the copy warp

// ------------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(saddr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(saddr(b)), "r"(bytes) : "memory");
}
// Test for completion of the phase with the given parity; the thread may sleep in
// the instruction meanwhile, for a system-dependent time (no hint: measured faster
// on the floodplain than a 0.1 ms or 1 us hint).
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Non-blocking test for completion of the phase with the given parity.
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase with the given parity to complete; false after ~1 s.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity) {
  if (mbar_try(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try(b, parity))
    if (clock64() - t0 > kWaitCycles) return false;
  return true;
}
// Bulk copy global -> shared (16-byte aligned, size a multiple of 16), completing on b.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   saddr(dst)),
               "l"(src), "r"(bytes), "r"(saddr(b))
               : "memory");
}
// Element copy global -> shared (N = 4 or 8 bytes, aligned to N).
template <int N>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(saddr(dst)), "l"(src), "n"(N) : "memory");
}
// Arrive on b once this thread's earlier cp.async copies have landed (the arrival is
// counted in b's expected count).
__device__ __forceinline__ void cp_async_arrive(uint64_t* b) {
  asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(saddr(b)) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// Programmatic dependent launch: wait until the previous kernel in the stream has
// completed and its memory is visible (returns at once without such a dependency);
// allow the next kernel to begin launching.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void grid_dep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

__device__ __forceinline__ bool is_zero(double x) { return (__double_as_longlong(x) << 1) == 0; }
__device__ __forceinline__ bool is_zero(float x) { return (__float_as_uint(x) << 1) == 0u; }
// h = H - z <= 0 for a cell (FP64: exact, from the keys; FP32-bulk: the pair's depth).
__device__ __forceinline__ bool cell_dry(double H, double, double z) { return okey(H) <= okey(z); }
__device__ __forceinline__ bool cell_dry(float hi, float lo, float z) { return !(depth_of(hi, lo, z) > 0.0f); }

// ------------------------------------------------------------------ shared memory

// Written by the copy warp next to a slot's group A, before the group's arrival.
struct StageInfo {
  int tile, ne, nh, inst;
  uint32_t flags;
  int bidx;       // rank among the instance's tiles with boundary edges
  int item;       // index of the work item
  int pad;
};
static_assert(sizeof(StageInfo) % 16 == 0, "the staged arrays after StageInfo take bulk copies (16-byte aligned)");

// Shared-memory layout of a step CTA with kS tile slots (the copy warp stages up to kS
// tiles ahead of the compute warps).
template <typename T, int kS = 3>
struct StepLayout {
  static constexpr bool k64 = sizeof(T) == 8;
  static constexpr int S = sizeof(T);
  static constexpr int kSlots = kS;
  static_assert(kS >= 2 && kS <= 4, "2 to 4 slots");
  static constexpr int kNA = k64 ? 4 : 5;  // staged per-cell arrays
  // array order: FP64 H qx qy z; FP32-bulk H Hlo qx qy z
  static constexpr int kH = 0, kHl = 1, kQx = k64 ? 1 : 2, kQy = k64 ? 2 : 3, kZ = k64 ? 3 : 4;
  static constexpr uint32_t kDesc = (sizeof(InstDesc<T>) + 15) & ~15u;
  static constexpr uint32_t kSlice = kTile * S;
  uint32_t ne4, nh4, nloc;
  uint32_t desc, ctl, info, arr, gn2, slot;  // within a slot (record at 0), slot size
  uint32_t F, uvc, dry, skip, red, elist, total;  // from the start of shared memory
  BM_HD StepLayout(uint32_t ne4_, uint32_t nh4_) {
    ne4 = ne4_;
    nh4 = nh4_;
    nloc = kTile + nh4;
    desc = align16(RecLayout<S>::bytes(ne4, nh4));
    ctl = desc + kDesc;
    info = ctl + static_cast<uint32_t>(sizeof(Ctl));
    arr = align16(info + static_cast<uint32_t>(sizeof(StageInfo)));  // bulk-copy destinations: 16-byte aligned
    gn2 = arr + kNA * nloc * S;
    slot = (gn2 + kSlice + 127u) & ~127u;
    F = kSlots * slot;
    // the flux arrays; also the finalize's 2 kTile partial sums (free at the end of a tile)
    uvc = F + (5 * ne4 * S > 2 * kTile * 8 ? 5 * ne4 * S : 2 * kTile * 8);
    dry = uvc + 3 * nloc * S;
    skip = dry + align16(nloc);
    red = skip + align16(ne4);
    elist = red + (4 + 24) * 8;  // finalize broadcast slots and reduction buffer
    total = elist + (k64 ? align16(2 * ne4) : 0u);  // FP64: phase F's list of edges with water
  }
};

// ------------------------------------------------------------------ the copy warp

// Lane l's source of a group-A state slice for an instance: lane 3 + j copies array j
// (order of StepLayout), lane 3 + kNA copies g n^2; read from the instance's
// descriptor in global memory at the parity of its control block.  Both buffers'
// pointers and the parity are read independently (one memory round trip).
template <typename P>
__device__ __forceinline__ P ldg_ptr(const P* p) {
  return reinterpret_cast<P>(__ldg(reinterpret_cast<const unsigned long long*>(p)));
}
template <typename T>
__device__ __forceinline__ const T* slice_src(const PipeItem& it, int lane) {
  using SL = StepLayout<T>;
  const InstDesc<T>* d = static_cast<const InstDesc<T>*>(it.desc);
  const int j = lane - 3;
  T* const* pair = nullptr;  // double-buffered arrays
  const T* const* one = nullptr;
  if constexpr (SL::k64) {
    pair = j == 0 ? d->H : j == 1 ? d->qx : j == 2 ? d->qy : nullptr;
    one = j == 3 ? &d->z : j == 4 ? &d->gn2 : nullptr;
  } else {
    pair = j == 0 ? d->H : j == 1 ? d->Hlo : j == 2 ? d->qx : j == 3 ? d->qy : nullptr;
    one = j == 4 ? &d->z : j == 5 ? &d->gn2 : nullptr;
  }
  if (one != nullptr) return ldg_ptr(one);
  if (pair == nullptr) return nullptr;
  const int par = it.ctl->parity;
  const T* p0 = ldg_ptr(pair);
  const T* p1 = ldg_ptr(pair + 1);
  return par ? p1 : p0;
}

// Group A of a tile into a slot (all lanes of the copy warp; src = this lane's slice
// source for the tile's instance).
template <typename T, int kS>
__device__ __forceinline__ void issue_a(const StepLayout<T, kS>& L, unsigned char* sa, const PipeItem& it, int item,
                                        const T* const* ssrc, uint64_t* mb, int lane) {
  using SL = StepLayout<T, kS>;
  if (lane == 0) {
    StageInfo* inf = reinterpret_cast<StageInfo*>(sa + L.info);
    inf->tile = it.tile;
    inf->ne = static_cast<int>(it.ne_nh & 0xffffu);
    inf->nh = static_cast<int>(it.ne_nh >> 16);
    inf->inst = it.inst;
    inf->flags = it.flags;
    inf->bidx = static_cast<int>(it.bidx);
    inf->item = item;
    // the arrival (release) orders the stores above before the phase completes
    mbar_expect_tx(mb, it.rec_bytes + SL::kDesc + static_cast<uint32_t>(sizeof(Ctl)) + (SL::kNA + 1) * SL::kSlice);
  }
  __syncwarp();
  if (lane == 0) {
    bulk_g2s(sa, it.rec, it.rec_bytes, mb);
  } else if (lane == 1) {
    bulk_g2s(sa + L.desc, it.desc, SL::kDesc, mb);
  } else if (lane == 2) {
    bulk_g2s(sa + L.ctl, it.ctl, static_cast<uint32_t>(sizeof(Ctl)), mb);
  } else if (lane <= 3 + SL::kNA) {
    const int j = lane - 3;
    unsigned char* dst = j < SL::kNA ? sa + L.arr + j * L.nloc * SL::S : sa + L.gn2;
    bulk_g2s(dst, ssrc[j] + static_cast<size_t>(it.tile) * kTile, SL::kSlice, mb);
  }
}

// The first kHaloPre halo indices of a tile, read from its record in global memory
// (lane l holds entries l, l + 32, l + 64), ahead of the tile's issue.
constexpr int kHaloPre = 3;
template <typename T>
__device__ __forceinline__ void load_halo(const PipeItem& it, int lane, int (&hv)[kHaloPre]) {
  const int nh = it.tile >= 0 ? static_cast<int>(it.ne_nh >> 16) : 0;
  const int32_t* hg =
      reinterpret_cast<const int32_t*>(it.rec + RecLayout<sizeof(T)>::hidx(round4(it.ne_nh & 0xffffu)));
#pragma unroll
  for (int u = 0; u < kHaloPre; ++u) {
    const int h = lane + 32 * u;
    hv[u] = h < nh ? __ldg(hg + h) : 0;
  }
}

// Group H of a tile (all lanes of the copy warp): the halo cells' values by cp.async,
// each lane arriving on mb when its gathers have landed.  ssrc: the instance's slice
// sources (shared memory, array j at j); hv: the prefetched halo indices.
template <typename T, int kS>
__device__ __forceinline__ void issue_h(const StepLayout<T, kS>& L, unsigned char* sa, const PipeItem& it,
                                        const T* const* ssrc, const int (&hv)[kHaloPre], uint64_t* mb, int lane) {
  using SL = StepLayout<T, kS>;
  const int nh = static_cast<int>(it.ne_nh >> 16);
  T* arr = reinterpret_cast<T*>(sa + L.arr);
#pragma unroll
  for (int j = 0; j < SL::kNA; ++j) {
    const T* sp = ssrc[j];
    T* dst = arr + j * L.nloc + kTile;
#pragma unroll
    for (int u = 0; u < kHaloPre; ++u) {
      const int h = lane + 32 * u;
      if (h < nh) cp_async<sizeof(T)>(dst + h, sp + hv[u]);
    }
  }
  if (nh > 32 * kHaloPre) {  // large halos (unusual meshes): the rest of the indices now
    const int32_t* hg =
        reinterpret_cast<const int32_t*>(it.rec + RecLayout<SL::S>::hidx(round4(it.ne_nh & 0xffffu)));
    for (int h = 32 * kHaloPre + lane; h < nh; h += 32) {
      const int gi = __ldg(hg + h);
#pragma unroll
      for (int j = 0; j < SL::kNA; ++j) cp_async<sizeof(T)>(arr + j * L.nloc + kTile + h, ssrc[j] + gi);
    }
  }
  cp_async_arrive(mb);
}

// ------------------------------------------------------------------ the step

// While the lists hold most items, every kProbe-th launch builds them again.
constexpr int kProbe = 16;

// A work list as the step kernel sees it.  sched (kSchedInts): [0] tickets handed out
// by the counter (after each CTA's static tickets), [1] CTAs done taking items (both
// zero at launch; the last CTA to finish taking zeroes them), [2] launch stamp s, [3]
// / [6] front / back items listed for launch s + 1, [4] / [7] the same listed for this
// launch, [8] what this launch takes: 1 the
// fixed and the listed items, 0 every item (FP64: the listed ones first), 2 every item
// in work-list order (the lists held most of them: they are built again only every
// kProbe-th launch, to see whether they still do), 3 every item in work-list order,
// building the lists (after a prime pass, whose lists hold every item: only one state
// buffer is valid then), [9] listing allowed (host-set),
// [10] / [11] (one 64-bit word) tickets accounted (items finished plus tickets skipped)
// / items finished in this launch, [12] items the previous launch finished.
// early: 2 x n_items, per stamp parity the listed items (front part from index 0 up,
// back part from the end down); mark: 2 x n_items, per stamp parity 2 s + 1 for an item
// listed in front for launch s, 2 s for one listed in back only (kFixedMark: a fixed
// item, never listed).  An item listed in back and then in front is in both parts; its
// back ticket skips it.
struct ListArgs {
  const PipeItem* items;
  int* sched;
  int* early;
  int* mark;
  const int* fixed;      // the fixed items (tile flags in kFixedFlags, and item 0)
  const int* inst_item;  // per instance: its first item
  int n_items, n_fixed, n_inst;
  int ne4max, nh4max;    // the largest record of the list (they fix the shared-memory layout)
  int lazy;              // claiming: 0 ahead; 1 the next item right after an issue (no lookahead);
                         // 2 each item once its slot is free; 3 also once the previous
                         // tile is past its edge phase
};

// A work list's scheduling state for a full launch: counters zero, listing allowed or
// not, no item listed, fixed items marked.
__global__ void list_reset(const PipeItem* items, int n_items, int* mark, int* sched, int listed_ok) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kSchedInts) sched[i] = i == 9 ? listed_ok : 0;
  if (i < n_items) {
    const int v = (i == 0 || (items[i].flags & kFixedFlags)) ? kFixedMark : -1;
    mark[i] = v;
    mark[n_items + i] = v;
  }
}

template <typename T>
constexpr int kMinBlocks = sizeof(T) == 8 ? 2 : 3;
// Share of a launch's tickets handed out statically: static16 / kStaticDen, by default
// kStaticNum; the autotuner searches it.
constexpr int kStaticDen = 16;
template <typename T>
constexpr int kStaticNum = sizeof(T) == 8 ? 0 : 4;  // measured over the 2M floodplain's run

// One step (prime = 0) or prime pass (prime = 1: no update; derived data, inflow
// weights and the dt of the current state) over a work list g.  Ticket t < F takes
// fixed[t]; F <= t < F + nf the front part of the listed items, then nb of the back
// part; a full launch then takes item t - E (E = F + nf + nb) unless it is fixed or was
// taken from the lists (its mark is s).  FP32-bulk full launches use no lists.  A
// single state is a list of one instance's tiles, so a run executes the same machine
// code alone and in a batch and gives bitwise the same result.  kX: which optional
// features the instantiation carries -- 0 none; 1 the flood-tracking records and the
// edge mass fluxes exported for passive species; 2 also external sources and the
// logarithmic friction closures (a list launches the lowest level its members need,
// so the plain step carries none of that code).  withhold != 0 (diagnostics of the
// failure path only): every CTA's copy warp withholds group H of its first tile, so
// the compute warps' bounded wait for it runs out; the launch then takes the timeout
// path below (status bit 2, issued copies retired, no state written).  static16: the
// static share of the tickets in sixteenths (negative: kStaticNum); the schedule never
// changes results (the reductions are order-free).  kS: the tile slots in shared memory
// (how far the copy warp may run ahead; the plain level is built for 2, 3 and 4 slots,
// the others for 3).
template <typename T, int kX, int kS = 3>
__global__ void __launch_bounds__(kStepThreads, kMinBlocks<T>) step_pipe(const ListArgs g, int prime, int withhold,
                                                                         int static16) {
  constexpr bool kExtra = kX >= 1;  // tracking, species exports
  constexpr bool kFull = kX >= 2;   // sources, log-law friction
  using SL = StepLayout<T, kS>;
  using RL = RecLayout<SL::S>;
  constexpr bool kPair = !SL::k64;
  constexpr int S = SL::kSlots;
  const PipeItem* __restrict__ items = g.items;
  int* __restrict__ sched = g.sched;
  int* __restrict__ early = g.early;
  int* __restrict__ mark = g.mark;
  const int n_items = g.n_items;
  extern __shared__ __align__(128) unsigned char smem[];
  // per slot: group A landed, group H landed, slot released by the compute warps
  __shared__ __align__(8) uint64_t mb_a[S], mb_h[S], mb_e[S];
  __shared__ int s_abort;
  // tiles whose edge phase the compute warps have finished (claiming mode 3 claims item
  // j only once tile j - 1 is past its edges: long tiles commit late, nearly greedily)
  __shared__ int s_edged;
  __shared__ int s_nact;  // FP64: the length of the phase F edge list
  // the launch's ticket map (written by the copy warp before its first issue, so the
  // compute warps see it after their first wait): stamp, listing allowed, part bounds
  // P1 <= P2 <= P3 <= tickets, whether the lists were taken; the tickets this CTA's copy
  // warp skipped (written before its end marker)
  __shared__ int s_stamp, s_listed_ok, s_order, s_p1, s_p2, s_p3, s_tickets, s_lists, s_skip;
  // the compute warps' listings (item * 2 + front), flushed to the next launch's list in
  // bulk (one round of atomics for many tiles, off the tiles' critical path); FP64 has
  // less shared memory to spare (two CTAs of its layout fill an SM)
  constexpr int kLstCap = SL::k64 ? 128 : 1024;
  __shared__ int s_lst[kLstCap];
  __shared__ int s_nlst;
  __shared__ int s_fin;  // the finalizes a tile's CTA runs (bit 0 boundary, bit 1 inflow)
  __shared__ __align__(16) PipeItem s_pa;  // the copy warp's next item to issue
  __shared__ const T* s_src[SL::kNA + 1];  // its instance's state slices' sources (arrays, then g n^2)
  const SL L(static_cast<uint32_t>(g.ne4max), static_cast<uint32_t>(g.nh4max));
  const int tid = threadIdx.x;
  auto slot = [&](int k) { return smem + (k % S) * L.slot; };

  if (tid == 0) {
    for (int s = 0; s < S; ++s) {
      mbar_init(&mb_a[s], 1);
      mbar_init(&mb_h[s], 32);
      mbar_init(&mb_e[s], kTile / 32);
    }
    mbar_init_fence();
    s_abort = 0;
    s_edged = 0;
    s_nlst = 0;
  }
  __syncthreads();

  if (tid >= kTile) {
    // ---------------------------------------------------------------- copy warp
    const int lane = tid - kTile;
    volatile int* abort_flag = &s_abort;
    // Work items reach the issue through a pipeline, so the copy warp seldom waits on a
    // value in the iteration that asked for it: the ticket (static, or requested from
    // the counter a step ahead) and its lookup -> the item read -> promotion to "next
    // to issue" (instance pointers and halo indices read) -> issue.
    // A work item read ahead is held across the warp, one 32-bit word of it per lane
    // (lanes 0..11; lane 12 holds its mark for a back-part item): the next to issue is
    // in shared memory (s_pa), so the copy warp keeps few registers.
    constexpr int kRest = 1 << 30, kBack = 1 << 29, kIdx = kBack - 1;
    constexpr int kWords = static_cast<int>(sizeof(PipeItem) / 4), kWTile = 7, kWInst = 9, kWFlags = 10;
    auto fetch_w = [&](int idx) -> unsigned {
      if (idx < 0) return lane == kWTile ? 0xffffffffu : 0u;  // tile -1: no item
      const int i = idx & kIdx;
      if (lane < kWords) return __ldg(reinterpret_cast<const unsigned*>(items + i) + lane);
      if (lane == kWords && (idx & kBack))
        return static_cast<unsigned>(__ldcg(&mark[static_cast<size_t>(s_stamp & 1) * n_items + i]));
      return 0u;
    };
    auto word = [&](unsigned w, int k) -> unsigned { return __shfl_sync(0xffffffffu, w, k); };
    const PipeItem& pa = s_pa;
    int hv_a[kHaloPre];
    // A CTA whose first ticket (its own index) is a fixed item reads that item and its
    // halo indices before the previous launch has ended (items and records do not
    // change) and issues it right after the wait.
    const int idx_early = static_cast<int>(blockIdx.x) < min(g.n_fixed, n_items) ? __ldg(&g.fixed[blockIdx.x]) : -1;
    if (idx_early >= 0) {
      const unsigned w = fetch_w(idx_early);
      if (lane < kWords) reinterpret_cast<unsigned*>(&s_pa)[lane] = w;
      __syncwarp();
      load_halo<T>(pa, lane, hv_a);
    }
    // The lists, the marks and the counters are the previous launch's.
    grid_dep_wait();
    // the early item's slice sources (its instance's buffer parity is the previous
    // launch's), loaded together with the counters below: one round trip, not two
    const T* src_early = idx_early >= 0 ? slice_src<T>(pa, lane) : nullptr;
    if (lane == 0) {
      const volatile int* vs = sched;
      const int stamp = vs[2], mode = vs[8];
      const bool listed = mode == 1;
      const int n_fix = min(g.n_fixed, n_items);
      // FP32-bulk full launches take the work list in order after the fixed items
      const bool use_lists = listed || (SL::k64 && mode == 0);
      const int nf = use_lists ? min(max(vs[4], 0), n_items - n_fix) : 0;
      const int nb = use_lists ? min(max(vs[7], 0), n_items - n_fix - nf) : 0;
      s_stamp = stamp;
      // listing: allowed, and (every item taken in work-list order) only on a probe
      s_listed_ok = vs[9] && !(mode == 2 && stamp % kProbe != kProbe - 1);  // (modes 2, 3: in work-list order)
      s_order = SL::k64 && !vs[9];  // FP64 without skipping: list the tiles that stepped, to take them first
      s_p1 = n_fix;
      s_p2 = n_fix + nf;
      s_p3 = n_fix + nf + nb;
      s_tickets = n_fix + nf + nb + (listed ? 0 : n_items);
      s_lists = nf + nb > 0;
    }
    __syncwarp();
    const int n_tickets = s_tickets;
    int n_skip = 0;  // tickets resolved to an item taken otherwise
    // ticket -> work item (-1: taken otherwise; -2: past the end), in two parts so the
    // load can be issued a step ahead: map_load reads what the ticket needs (a fixed or
    // listed item, or the item's mark), resolve decides.
    auto map_load = [&](int t) -> int {
      const int p1 = s_p1, p2 = s_p2, p3 = s_p3;
      const size_t par = static_cast<size_t>(s_stamp & 1) * n_items;
      if (t < p1) return __ldg(&g.fixed[t]);
      if (t < p2) return __ldcg(&early[par + (t - p1)]);
      if (t < p3) return __ldcg(&early[par + (n_items - 1 - (t - p2))]);
      if constexpr (SL::k64) {
        if (t < n_tickets) return __ldcg(&mark[par + (t - p3)]);
      }
      return 0;
    };
    // Index flags checked once the item is read: kRest, an FP32-bulk full launch takes
    // item t - P3 without a lookup and skips it if it is a fixed one (taken by a ticket
    // t < P1); kBack, an item of the list's back part is skipped if it is in the front
    // part too (its mark, read with the item, says so)
    auto resolve = [&](int t, int v) -> int {
      const int p2 = s_p2, p3 = s_p3;
      if (t < p3) return (v >= 0 && v < n_items) ? (t < p2 ? v : v | kBack) : -1;  // (valid lists hold valid items)
      if (t >= n_tickets) return -2;
      if constexpr (SL::k64) {
        if (v == kFixedMark || (s_lists && (v >> 1) == s_stamp)) return -1;
        return t - p3;
      } else {
        return (t - p3) | kRest;
      }
    };
    auto taken_otherwise = [&](int idx, unsigned w) -> bool {
      const unsigned fl = word(w, kWFlags);
      const int m = static_cast<int>(word(w, kWords));
      if (idx < 0) return false;
      if (idx & kRest) return (idx & kIdx) == 0 || (fl & kFixedFlags) != 0u;
      return (idx & kBack) != 0 && m == 2 * s_stamp + 1;
    };
    // Tickets: first this CTA's static ones, blockIdx.x + m gridDim.x for m < m_static
    // (known without asking, so their items are looked up ahead -- the first 32 in one
    // round at the start -- without waiting; a share of all tickets, so that the
    // counter's rest evens out the CTAs), then the launch's counter from n_static on,
    // one ticket requested a step ahead.
    // A CTA's tickets increase, so once one is past the end every later one is too.
    const int G = static_cast<int>(gridDim.x);
    const int m_static =
        max(g.lazy ? 1 : 2, n_tickets / kStaticDen * (static16 >= 0 ? static16 : kStaticNum<T>) / G);
    const int n_static = m_static * G;
    const int pre_v = lane < m_static ? map_load(static_cast<int>(blockIdx.x) + lane * G) : 0;
    int m_next = idx_early >= 0 ? 1 : 0;  // (the early item was ticket 0)
    int tc = 0;  // lane 0: the requested counter ticket
    bool tc_pending = false;
    auto request = [&]() {
      if (lane == 0) tc = atomicAdd(&sched[0], 1) + n_static;
      tc_pending = true;
    };
    auto next_tv = [&](int& v) -> int {  // the next ticket and its lookup
      if (m_next < m_static) {
        const int m = m_next++;
        const int pv = __shfl_sync(0xffffffffu, pre_v, m & 31);
        const int t = static_cast<int>(blockIdx.x) + m * G;
        v = m < 32 ? pv : map_load(t);
        return t;
      }
      if (!tc_pending) request();
      tc_pending = false;
      const int t = __shfl_sync(0xffffffffu, tc, 0);
      v = map_load(t);
      return t;
    };
    auto next_idx = [&]() -> int {  // the next ticket's item, past skipped tickets (waits)
      int idx;
      do {
        int v;
        const int t = next_tv(v);
        idx = resolve(t, v);
        if (idx == -1) ++n_skip;
      } while (idx == -1);
      return idx;
    };
    // start-up: item a (next to issue) and item b (read), read together -- or, after
    // an early item a, b once a is issued
    int idx_a = idx_early, idx_b = -2;
    unsigned wb = fetch_w(-2);
    // claiming on demand (lazy 2): a is claimed and read once its slot is free, so
    // b_pending says a is still to be claimed; otherwise it says b is still to be read
    const bool on_demand = g.lazy >= 2;
    const bool gated = g.lazy == 3;
    const volatile int* edged = &s_edged;
    bool b_pending = on_demand ? idx_early < 0 : idx_early >= 0;
    if (!on_demand && !b_pending) {
      idx_a = next_idx();
      idx_b = idx_a >= 0 ? next_idx() : -2;
      unsigned wa = fetch_w(idx_a);
      wb = fetch_w(idx_b);
      while (taken_otherwise(idx_a, wa)) {
        ++n_skip;
        idx_a = idx_b;
        wa = wb;
        idx_b = idx_a >= 0 ? next_idx() : -2;
        wb = fetch_w(idx_b);
      }
      if (lane < kWords) reinterpret_cast<unsigned*>(&s_pa)[lane] = wa;
      __syncwarp();
      load_halo<T>(pa, lane, hv_a);
    }
    bool tc_live = false;
    int tn = -2, tv = 0;  // the ticket after b and its lookup, resolved at the promotion
    auto lookahead = [&]() {
      tc_live = idx_b >= 0 && !g.lazy;
      if (tc_live) {
        tn = next_tv(tv);
        if (m_next >= m_static && !tc_pending) request();
      }
    };
    if (!on_demand && !b_pending) lookahead();
    // the slice sources of a's instance (lane 3 + j reads array j's)
    auto set_src = [&]() {
      const T* p = slice_src<T>(pa, lane);
      if (lane >= 3 && lane <= 3 + SL::kNA) s_src[lane - 3] = p;
      __syncwarp();
    };
    int src_inst = -1;  // the instance whose slice sources s_src holds
    if (idx_early >= 0) {
      if (lane >= 3 && lane <= 3 + SL::kNA) s_src[lane - 3] = src_early;
      __syncwarp();
      src_inst = pa.inst;
    } else if (!on_demand && pa.tile >= 0) {
      set_src();
      src_inst = pa.inst;
    }
    int a_next = 0;      // next tile (in this CTA's order) whose groups are issued
    bool ended = false;  // the end marker has been issued
    long long idle0 = clock64();
    bool ok = true;
    while (!ended) {
      bool progress = false;
      // groups A and H of the next tile (or the end marker) once its slot is free
      bool free_slot = a_next < S;
      if (!free_slot && lane == 0) free_slot = mbar_test(&mb_e[a_next % S], ((a_next - S) / S) & 1);
      if (gated && a_next > 0 && lane == 0) free_slot = free_slot && *edged >= a_next;
      if (__shfl_sync(0xffffffffu, free_slot, 0)) {
        if (on_demand && b_pending) {
          // the item for this slot: claimed, read and promoted now
          b_pending = false;
          int idx = next_idx();
          unsigned w = fetch_w(idx);
          while (taken_otherwise(idx, w)) {
            ++n_skip;
            idx = next_idx();
            w = fetch_w(idx);
          }
          const int w_tile = static_cast<int>(word(w, kWTile)), w_inst = static_cast<int>(word(w, kWInst));
          __syncwarp();  // every lane is done with the previous item
          if (lane < kWords) reinterpret_cast<unsigned*>(&s_pa)[lane] = w;
          __syncwarp();
          if (w_tile >= 0 && w_inst != src_inst) {
            set_src();
            src_inst = w_inst;
          }
          idx_a = idx;
          load_halo<T>(pa, lane, hv_a);
        }
        if (pa.tile >= 0 && on_demand) {
          issue_a<T>(L, slot(a_next), pa, idx_a & kIdx, s_src, &mb_a[a_next % S], lane);
          if (!(withhold && a_next == 0)) issue_h<T>(L, slot(a_next), pa, s_src, hv_a, &mb_h[a_next % S], lane);
          b_pending = true;  // the next item once the next slot is free
        } else if (pa.tile >= 0) {
          issue_a<T>(L, slot(a_next), pa, idx_a & kIdx, s_src, &mb_a[a_next % S], lane);
          if (!(withhold && a_next == 0)) issue_h<T>(L, slot(a_next), pa, s_src, hv_a, &mb_h[a_next % S], lane);
          if (b_pending) {  // after an early item a, or (claiming lazily) every issue
            b_pending = false;
            idx_b = next_idx();
            wb = fetch_w(idx_b);
            lookahead();
          }
          while (taken_otherwise(idx_b, wb)) {  // b was taken otherwise: the one after it
            ++n_skip;
            int idx = tc_live ? resolve(tn, tv) : (g.lazy ? next_idx() : -2);
            if (idx == -1) {
              ++n_skip;
              idx = next_idx();
            }
            idx_b = idx;
            wb = fetch_w(idx_b);
            tc_live = idx_b >= 0 && !g.lazy;
            if (tc_live) {
              tn = next_tv(tv);
              if (m_next >= m_static && !tc_pending) request();
            }
          }
          const int b_tile = static_cast<int>(word(wb, kWTile)), b_inst = static_cast<int>(word(wb, kWInst));
          // promote b (read one iteration ago); read its instance pointers and halo
          // indices (used at the next issue)
          const int a_inst = pa.inst;
          __syncwarp();  // every lane is done with a
          if (lane < kWords) reinterpret_cast<unsigned*>(&s_pa)[lane] = wb;
          __syncwarp();
          if (b_tile >= 0 && b_inst != a_inst) set_src();
          idx_a = idx_b;
          load_halo<T>(pa, lane, hv_a);
          // the pending ticket becomes the next read; request a new ticket
          if (b_tile >= 0 && tc_live) {
            // the ticket looked up a step ago; past a skipped one, the next ones now
            int idx = resolve(tn, tv);
            if (idx == -1) {
              ++n_skip;
              idx = next_idx();
            }
            idx_b = idx;
            wb = fetch_w(idx_b);  // used at the next promotion: its load is not waited for here
            tc_live = idx_b >= 0;
            if (tc_live) {
              tn = next_tv(tv);
              if (m_next >= m_static && !tc_pending) request();
            }
          } else {
            wb = fetch_w(-2);
            idx_b = -2;
            tc_live = false;
            b_pending = g.lazy && b_tile >= 0;  // claiming lazily: the next item at the next issue
          }
        } else {
          if (lane == 0) {
            reinterpret_cast<StageInfo*>(slot(a_next) + L.info)->tile = -1;
            s_skip = n_skip;  // released to the compute warps by the arrival below
            mbar_expect_tx(&mb_a[a_next % S], 0);
          }
          cp_async_arrive(&mb_h[a_next % S]);  // end marker: nothing to gather
          ended = true;
          grid_dep_launch();  // this CTA takes no more items
        }
        ++a_next;
        progress = true;
      }
      if (progress) {
        idle0 = clock64();
      } else {
        if (*abort_flag || clock64() - idle0 > kWaitCycles) {
          ok = false;
          break;
        }
        __nanosleep(100);
      }
    }
    cp_async_wait_all();
    if (lane == 0) {
      if (!ok) {
        *abort_flag = 1;
        atomicOr(&items[0].ctl->status, 4);
      }
      // every CTA takes exactly one item past the end (or gives up); the last to do so
      // zeroes the counters for the next launch
      if (atomicAdd(&sched[1], 1) == static_cast<int>(gridDim.x) - 1) {
        atomicExch(&sched[0], 0);
        atomicExch(&sched[1], 0);
      }
    }
    if (!ok) {
      // let the bulk copies of the groups issued land before the CTA exits
      for (int j = a_next - 1; j >= 0 && j >= a_next - S; --j) (void)mbar_wait(&mb_a[j % S], (j / S) & 1);
    }
    return;
  }

  // ------------------------------------------------------------------ compute warps
  grid_dep_wait();
  T* Fs = reinterpret_cast<T*>(smem + L.F);
  unsigned char* dry = smem + L.dry;
  unsigned char* skip = smem + L.skip;
  double* red = reinterpret_cast<double*>(smem + L.red);
  const T zero = T(0);
  volatile int* abort_flag = &s_abort;
  // list an item for the next launch, once per part (its mark: 2 s1 + 1 in front, 2 s1
  // in back; a back listing after a front one adds nothing)
  auto list_next = [&](int item, bool front) {
    const int s1 = s_stamp + 1;
    const size_t par = static_cast<size_t>(s1 & 1) * n_items;
    const int v = 2 * s1 + (front ? 1 : 0);
    if (item < 0 || item >= n_items || atomicMax(&mark[par + item], v) >= v) return;
    const int pos = atomicAdd(&sched[front ? 3 : 6], 1);
    if (pos < n_items) early[par + (front ? pos : n_items - 1 - pos)] = item;
  };
  // note a listing in the CTA's buffer (at once when the buffer is full)
  auto note = [&](int item, bool front) {
    const int pos = atomicAdd(&s_nlst, 1);
    if (pos < kLstCap) s_lst[pos] = item * 2 + (front ? 1 : 0);
    else list_next(item, front);
  };
  // the buffer's listings, all compute threads: dedupe by the marks, then one counter
  // add per warp and part
  auto flush = [&]() {
    nbar<kTile>();
    const int n = min(s_nlst, kLstCap);
    const int s1 = s_stamp + 1;
    const size_t par = static_cast<size_t>(s1 & 1) * n_items;
    const int lane = tid & 31;
    for (int b0 = 0; b0 < n; b0 += kTile) {
      const int j = b0 + tid;
      int item = -1;
      bool front = false, ok = false;
      if (j < n) {
        const int e = s_lst[j];
        item = e >> 1;
        front = (e & 1) != 0;
        const int v = 2 * s1 + (front ? 1 : 0);
        ok = item >= 0 && item < n_items && atomicMax(&mark[par + item], v) < v;
      }
      const unsigned mf = __ballot_sync(0xffffffffu, ok && front), mb = __ballot_sync(0xffffffffu, ok && !front);
      int bf = 0, bb = 0;
      if (lane == 0) {
        if (mf) bf = atomicAdd(&sched[3], __popc(mf));
        if (mb) bb = atomicAdd(&sched[6], __popc(mb));
      }
      bf = __shfl_sync(0xffffffffu, bf, 0);
      bb = __shfl_sync(0xffffffffu, bb, 0);
      if (ok) {
        const unsigned lt = (1u << lane) - 1u;
        const int pos = front ? bf + __popc(mf & lt) : bb + __popc(mb & lt);
        if (pos < n_items) early[par + (front ? pos : n_items - 1 - pos)] = item;
      }
    }
    nbar<kTile>();
    if (tid == 0) s_nlst = 0;
    nbar<kTile>();
  };
  // this CTA's max Eq. 21 rate over the current instance's tiles, in the working
  // precision (FP32-bulk: no FP64 instruction per cell; the max of the floats, converted
  // once, equals the max of the converted values)
  T rrun = T(0);
  float smax = 0.0f;  // FP64: the largest rate screen this lane's warp has seen for the instance
  unsigned cnt = 0;   // tiles of the current instance this CTA completed
  int cur_inst = -1;  // the instance of those tiles
  Ctl* cur_ctl = nullptr;
  // the CTA's rate max of an instance to its control block, when the CTA moves on to
  // another instance's tiles or has no more (all compute threads)
  auto flush_rate = [&]() {
    const double r = block_max_nonneg_all<kTile>(static_cast<double>(rrun), reinterpret_cast<unsigned long long*>(red));
    if (tid == 0 && r > 0.0) atomicMax(&cur_ctl->rmax_bits, static_cast<unsigned long long>(__double_as_longlong(r)));
    rrun = T(0);
    smax = 0.0f;
    cnt = 0;
  };
  int n_done = 0;     // items this CTA completed in the launch
  for (int k = 0;; ++k) {
    unsigned char* sb = slot(k);
    {
      const bool ok = mbar_wait(&mb_a[k % S], (k / S) & 1) && mbar_wait(&mb_h[k % S], (k / S) & 1);
      if (nbar_or<kTile>(!ok || *abort_flag)) {
        if (tid == 0) {
          *abort_flag = 1;
          atomicOr(&items[0].ctl->status, 4);
        }
        return;
      }
    }
    if (reinterpret_cast<const StageInfo*>(sb + L.info)->tile < 0) break;  // no more tiles

    const StageInfo& inf = *reinterpret_cast<const StageInfo*>(sb + L.info);
    const InstDesc<T>& a = *reinterpret_cast<const InstDesc<T>*>(sb + L.desc);
    const Ctl& cs = *reinterpret_cast<const Ctl*>(sb + L.ctl);
    const int tile = inf.tile, ne = inf.ne, nh = inf.nh;
    const uint32_t ne4 = round4(static_cast<uint32_t>(ne));
    const T* sIA = reinterpret_cast<const T*>(sb + RL::ia());
    const uint32_t* sSlot = reinterpret_cast<const uint32_t*>(sb + RL::slot());
    const uint32_t* sLR = reinterpret_cast<const uint32_t*>(sb + RL::lr());
    const T* sNx = reinterpret_cast<const T*>(sb + RL::nx(ne4));
    const T* sNy = reinterpret_cast<const T*>(sb + RL::ny(ne4));
    const T* sLn = reinterpret_cast<const T*>(sb + RL::len(ne4));
    const T* arr = reinterpret_cast<const T*>(sb + L.arr);
    const T* sH = arr + SL::kH * L.nloc;
    const T* sHl = arr + SL::kHl * L.nloc;  // FP32-bulk only
    const T* sQx = arr + SL::kQx * L.nloc;
    const T* sQy = arr + SL::kQy * L.nloc;
    const T* sZ = arr + SL::kZ * L.nloc;
    const T* sGn2 = reinterpret_cast<const T*>(sb + L.gn2);
    T* U = reinterpret_cast<T*>(smem + L.uvc);
    T* V = U + L.nloc;
    T* C = V + L.nloc;
    const bool run = prime || cs.active;
    if (inf.inst != cur_inst) {  // (every compute thread reads the same slot)
      if (cnt > 0) flush_rate();
      cur_inst = inf.inst;
      cur_ctl = a.ctl;
    }
    T dt, quni, g, hg, hmin;
    step_consts(&cs, a.p, dt, quni, g, hg, hmin);
    const double qscale = cs.qscale;
    const int wpos = cs.wpos;
    const int par = cs.parity;

    // phase D: wet/dry flags, velocity and celerity of tile and halo cells.
    // A tile whose cells and halo cells are all dry, whose cells are at rest and which
    // has no inflow edge is quiet: every flux is zero and U^{n+1} = U^n.
    if (SL::k64 && tid == 0) s_nact = 0;  // the phase F edge list (read before the last barrier)
    bool tq = true;
    if (run) {
      for (int j = tid; j < kTile + nh; j += kTile) {
        const T Hj = sH[j], Hlj = kPair ? sHl[j] : zero, zj = sZ[j];
        const bool dj = cell_dry(Hj, Hlj, zj);
        dry[j] = dj ? 1 : 0;
        tq = tq && dj && (j >= kTile || (is_zero(sQx[j]) && is_zero(sQy[j])));
        T u = zero, v = zero, c = zero;  // dry: at rest, zero celerity
        if (!dj) cell_derived<T>(depth_of(Hj, Hlj, zj), sQx[j], sQy[j], hmin, g, u, v, c);
        U[j] = u;
        V[j] = v;
        C[j] = c;
      }
    }
    // (no inflow or source; a level edge under a series may flood a dry tile)
    const bool quiet = nbar_and<kTile>(tq) && !prime && !(inf.flags & 6u) && !(kFull && (inf.flags & 32u) && a.zh_n > 0);
    if (s_nlst > kLstCap / 2) flush();  // (every compute thread reads the count after the barrier)

    // phase F: edges
    if (run && !prime && !quiet) {
      int nact = ne;  // the edges the flux loop visits (FP64: the list's length)
      const uint16_t* elist = reinterpret_cast<const uint16_t*>(smem + L.elist);
      if constexpr (SL::k64) {
        // FP64: the edges with water on a side, and inflow edges, are listed first and
        // the flux loop runs over that list, so that at a wet/dry front a warp's FP64
        // instructions run with all lanes busy (the list's order is free: each edge
        // writes its own slots).  The other edges take their zero fluxes here.
        uint16_t* list = reinterpret_cast<uint16_t*>(smem + L.elist);
        const int lane = tid & 31;
        for (int kb = 0; kb < ne; kb += kTile) {
          const int k2 = kb + tid;
          bool act = false;
          if (k2 < ne) {
            const uint32_t lr = sLR[k2];
            const int lL = static_cast<int>(lr & (kMaxLocal - 1));
            const int R = static_cast<int32_t>(lr) >> kLocBits;
            const int lR = R >= 0 ? R : lL;
            const bool inflow = R <= kInflow && kInflow - R < a.n_inflow;
            act = !(dry[lL] && dry[lR]) || inflow;
            if (!act) {
              Fs[k2] = zero;
              Fs[L.ne4 + k2] = zero;
              Fs[2 * L.ne4 + k2] = zero;
              Fs[3 * L.ne4 + k2] = zero;
              Fs[4 * L.ne4 + k2] = zero;
              skip[k2] = 1;
              if constexpr (kExtra) {
                if (a.ex_flux != nullptr) {
                  const size_t o = static_cast<size_t>(tile) * static_cast<size_t>(a.ex_stride) + k2;
                  a.ex_flux[o] = zero;
                  a.ex_right[o] = 0;
                }
              }
            }
          }
          const unsigned m = __ballot_sync(0xffffffffu, act);
          int base = 0;
          if (lane == 0 && m != 0u) base = atomicAdd(&s_nact, __popc(m));
          base = __shfl_sync(0xffffffffu, base, 0);
          if (act) list[base + __popc(m & ((1u << lane) - 1u))] = static_cast<uint16_t>(k2);
        }
        nbar<kTile>();
        nact = *reinterpret_cast<volatile int*>(&s_nact);
      }
      for (int j = tid; j < nact; j += kTile) {
        const int k2 = SL::k64 ? static_cast<int>(elist[j]) : j;
        const uint32_t lr = sLR[k2];
        const int lL = static_cast<int>(lr & (kMaxLocal - 1));
        const int R = static_cast<int32_t>(lr) >> kLocBits;
        const int lR = R >= 0 ? R : lL;
        const bool listed = R <= kInflow;  // an edge with a boundary law
        const bool inflow = listed && kInflow - R < a.n_inflow;
        const bool outflow = listed && !inflow;  // h-Q relation or weir
        T f0 = zero, f1 = zero, f2 = zero, f3 = zero, f4 = zero;
        bool right = false;  // the contact's right side is upwind (passive species)
        unsigned char skipped = 1;
        if (!(dry[lL] && dry[lR]) || inflow) {
          const T HLh = sH[lL], HLl = kPair ? sHl[lL] : zero, zL = sZ[lL];
          T HRh = HLh, HRl = HLl, zR = zL;
          if (R >= 0) {
            HRh = sH[lR];
            HRl = kPair ? sHl[lR] : zero;
            zR = sZ[lR];
          }
          // modified states (hydrostatic reconstruction on the higher bed)
          const T zs = dmax(zL, zR);
          const T h1 = pos(depth_of(HLh, HLl, zs));
          const T h2 = pos(depth_of(HRh, HRl, zs));
          if (gt0(h1) || gt0(h2) || inflow) {
            skipped = 0;
            const T nx = sNx[k2], ny = sNy[k2], l = sLn[k2];
            const T uL = U[lL], vL = V[lL], cL = C[lL];
            const T unL = uL * nx + vL * ny, utL = -uL * ny + vL * nx;
            T un2, ut2, c1, c2;
            if (R >= 0) {
              const T uR = U[lR], vR = V[lR], cR = C[lR];
              // the side with the higher bed keeps its own depth, hence its own celerity
              const bool lhi = !gt(zR, zL);  // zL >= zR
              const T clo = f_sqrt(g * (lhi ? h2 : h1));
              c1 = lhi ? cL : clo;
              c2 = lhi ? clo : cR;
              un2 = uR * nx + vR * ny;
              ut2 = -uR * ny + vR * nx;
            } else {
              c1 = cL;
              c2 = cL;
              // wall: mirrored normal velocity (so also an outflow edge, a wall while it
              // lets nothing out)
              un2 = (R == kWall || outflow) ? -unL : unL;
              ut2 = utL;
            }
            T F0, F1, F2, pL, pR;
            hllc<T>(h1, unL, utL, c1, h2, un2, ut2, c2, hg, F0, F1, F2, pL, pR, right);
            T GL = F1 - pL;
            const T GR = F1 - pR;
            if (R == kWall || outflow) {
              F0 = zero;  // impermeable, frictionless (an outflow edge's law: below)
              F2 = zero;
            } else if (inflow) {
              const int j = kInflow - R;
              const T q = wpos ? static_cast<T>(qscale * static_cast<double>(a.in_pw[j])) : quni;
              if (q > zero) {
                const T hcr = f_cbrt(f_div(q * q, g));
                const T hb = fmax(h1, hcr);
                F0 = -q;
                GL = f_div(q * q, hb) + hg * hb * hb - pL;
              } else {
                F0 = zero;
                GL = zero;
              }
              F2 = zero;
            }
            f0 = l * F0;
            f1 = l * (GL * nx - F2 * ny);
            f2 = l * (GL * ny + F2 * nx);
            f3 = l * (GR * nx - F2 * ny);
            f4 = l * (GR * ny + F2 * nx);
          }
        }
        Fs[k2] = f0;
        Fs[L.ne4 + k2] = f1;
        Fs[2 * L.ne4 + k2] = f2;
        Fs[3 * L.ne4 + k2] = f3;
        Fs[4 * L.ne4 + k2] = f4;
        skip[k2] = skipped;
        if constexpr (kExtra) {
          // passive species: this edge's l F_h (inflow: l (-q); 0 on walls and skipped
          // edges) and its upwind side, for the species kernel after the step
          if (a.ex_flux != nullptr) {
            const size_t o = static_cast<size_t>(tile) * static_cast<size_t>(a.ex_stride) + k2;
            a.ex_flux[o] = f0;
            a.ex_right[o] = right ? 1 : 0;
          }
        }
      }
      if (SL::k64 && kFull && (inf.flags & 56u)) nbar<kTile>();  // the boundary-law loop below revisits edges by owner
      if (kFull && (inf.flags & 56u)) {
        // outflow edges (h-Q relation, weir) and water-level edges, walls above: where
        // the law lets water out, the flux of the boundary state on the cell's outgoing
        // characteristic that carries it; under a level series, HLLC between the cell
        // and the level's boundary state (each thread revisits its own edges; states
        // with such laws run the full instantiation)
        const int j_level = a.n_inflow + a.n_hq + a.n_weir;
        T zh_hi = zero, zh_lo = zero;  // Z_b(t^n)
        if ((inf.flags & 32u) && a.zh_n > 0) level_pair<T>(a, cs.t, zh_hi, zh_lo);
        for (int k2 = tid; k2 < ne; k2 += kTile) {
          const uint32_t lr = sLR[k2];
          const int R = static_cast<int32_t>(lr) >> kLocBits;
          const int lL = static_cast<int>(lr & (kMaxLocal - 1));
          if (R > kInflow || kInflow - R < a.n_inflow) continue;
          const int j = kInflow - R;
          const T HLh = sH[lL], HLl = kPair ? sHl[lL] : zero, zL = sZ[lL];
          const T h1 = fmax(zero, depth_of(HLh, HLl, zL));
          const T nx = sNx[k2], ny = sNy[k2], l = sLn[k2];
          const T unL = U[lL] * nx + V[lL] * ny, utL = -U[lL] * ny + V[lL] * nx;
          if (j >= j_level) {
            if (a.zh_n == 0) continue;  // a wall until a series is set
            T hb, ub, cb;
            level_state<T>(zh_hi, zh_lo, zL, h1, unL, g, hmin, hb, ub, cb);
            if (!(gt0(h1) || gt0(hb))) continue;  // dry on both sides: no flux
            T F0, F1, F2, pL, pR;
            bool right = false;
            hllc<T>(h1, unL, utL, C[lL], hb, ub, utL, cb, hg, F0, F1, F2, pL, pR, right);
            const T GL = F1 - pL;
            Fs[k2] = l * F0;
            Fs[L.ne4 + k2] = l * (GL * nx - F2 * ny);
            Fs[2 * L.ne4 + k2] = l * (GL * ny + F2 * nx);
            skip[k2] = 0;
            if constexpr (kExtra) {
              if (a.ex_flux != nullptr) {
                const size_t o = static_cast<size_t>(tile) * static_cast<size_t>(a.ex_stride) + k2;
                a.ex_flux[o] = l * F0;
                a.ex_right[o] = right ? 1 : 0;
              }
            }
            continue;
          }
          if (dry[lL]) continue;
          T q = j < a.n_inflow + a.n_hq ? a.in_pw[j] : weir_discharge<T>(a, HLh, HLl, zL, h1, hmin);
          const T hb = q > zero ? outflow_state<T>(h1, unL, g, q) : T(-1);
          if (hb > zero) {
            const T GL = q * (q / hb) + hg * hb * hb - hg * h1 * h1;
            const T F2 = q * utL;
            Fs[k2] = l * q;
            Fs[L.ne4 + k2] = l * (GL * nx - F2 * ny);
            Fs[2 * L.ne4 + k2] = l * (GL * ny + F2 * nx);
            skip[k2] = 0;
            if constexpr (kExtra) {
              if (a.ex_flux != nullptr)
                a.ex_flux[static_cast<size_t>(tile) * static_cast<size_t>(a.ex_stride) + k2] = l * q;
            }
          }
        }
      }
    }
    if constexpr (kExtra) {
      // passive species: whether this tile exported fluxes (a quiet tile has none) and,
      // from tile 0, the step's dt (-1: the instance did not step)
      if (tid == 0 && a.ex_flux != nullptr && !prime) {
        a.ex_valid[tile] = (run && !quiet) ? 1 : 0;
        if (tile == 0) *a.ex_dt = run ? static_cast<double>(cs.dt) : -1.0;
      }
    }
    nbar<kTile>();
    if (tid == 0) *reinterpret_cast<volatile int*>(&s_edged) = k + 1;

    // phase I: cells
    const int i = tile * kTile + tid;
    if (run && i < a.n_cells) {
      T Hh = sH[tid], Hl = kPair ? sHl[tid] : zero;
      const T zi = sZ[tid], qxi = sQx[tid], qyi = sQy[tid], ia = sIA[tid], gn2 = sGn2[tid];
      const uint32_t sl = sSlot[tid];
      int idx[3], side[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        idx[q] = static_cast<int>((sl >> (kLocBits * q)) & (kMaxLocal - 1));
        side[q] = (sLR[idx[q]] & (kMaxLocal - 1)) != static_cast<uint32_t>(tid) ? 1 : 0;
      }
      const int dst = par ^ 1;
      int src = -1;  // the cell's source region
      if constexpr (kFull) {
        if (a.src_reg != nullptr) src = a.src_reg[i];
      }
      if (quiet || (src < 0 && !prime && skip[idx[0]] && skip[idx[1]] && skip[idx[2]] && dry[tid] && is_zero(qxi) &&
                    is_zero(qyi))) {
        // no flux, dry and at rest: U^{n+1} = U^n, velocity and celerity zero
        a.H[dst][i] = Hh;
        if constexpr (kPair) a.Hlo[dst][i] = Hl;
        a.qx[dst][i] = zero;
        a.qy[dst][i] = zero;
        if constexpr (kFull) {
          // a level edge's rate of Eq. 21 under the level of t^{n+1} (it may have risen
          // above the bed)
          if ((inf.flags & 32u) && a.zh_n > 0) {
            T zh_hi, zh_lo;
            level_pair<T>(a, prime ? cs.t : new_time(cs, 1), zh_hi, zh_lo);
            rrun = fmax(rrun, level_rate<T>(a, sLR, sNx, sNy, sLn, idx, zh_hi, zh_lo, zi, depth_of(Hh, Hl, zi), zero,
                                            zero, ia));
          }
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int code = static_cast<int32_t>(sLR[idx[q]]) >> kLocBits;
          if (code <= kInflow && kInflow - code < a.n_inflow) {
            a.in_pw[kInflow - code] = zero;
            a.in_hs[kInflow - code] = zero;
          }
        }
      } else {
        T h = depth_of(Hh, Hl, zi), ux = qxi, uy = qyi;
        if (!prime) {
          // flood tracking: the cell's record, loaded ahead of the update (a cell
          // copied through, dry and at rest, cannot change its record)
          bool trk = false;
          TrackRecord<T> rec{};
          if constexpr (kExtra) {
            trk = a.trk_t != nullptr;
            if (trk) rec = track_load(a, i);
          }
          T s0 = zero, s1 = zero, s2 = zero;
#pragma unroll
          for (int q = 0; q < 3; ++q) {
            const int e = idx[q];
            if (side[q] == 0) {
              s0 += Fs[e];
              s1 += Fs[L.ne4 + e];
              s2 += Fs[2 * L.ne4 + e];
            } else {
              s0 += -Fs[e];
              s1 += -Fs[3 * L.ne4 + e];
              s2 += -Fs[4 * L.ne4 + e];
            }
          }
          const T r = dt * ia;
          if constexpr (kPair) {
            pair_add(Hh, Hl, -(r * s0));
          } else {
            Hh = Hh - r * s0;
          }
          ux = qxi - r * s1;
          uy = qyi - r * s2;
          if constexpr (kFull) {
            // external source / sink, explicit in continuity (the S term of Eq. 12)
            if (src >= 0) {
              const T add = dt * a.src_rate[src];
              const int md = a.src_mode[src];
              if (md == 2 || (md == 1 && depth_of(Hh, Hl, zi) + add < zero)) {
                Hh = zi;  // the sink empties the cell
                if constexpr (kPair) Hl = zero;
              } else if constexpr (kPair) {
                pair_add(Hh, Hl, add);
              } else {
                Hh = Hh + add;
              }
            }
          }
          h = depth_of(Hh, Hl, zi);
          if (gt(h, hmin) && gt0(gn2)) {
            // split friction: two semi-implicit stages, Heun average.  With
            // a = dt k(q*), k(q) = g n^2 |q| / h^(7/3): q1 = q* / (1 + a), and since
            // |q1| = |q*| / (1 + a), q2 = q1 / (1 + dt k(q1)) = q* / (1 + 2a); so
            // (q* + q2) / 2 = q* (1 + a) / (1 + 2a) -- one square root and one
            // division instead of two each (equal up to rounding)
            T cf;  // k(q) / |q|: g n^2 / h^(7/3) (Manning), 1 / (h c_f)^2 (Table 1's log laws)
            bool manning = true;
            if constexpr (kFull) manning = a.fr_law == 0;
            if (manning) {
              const T r3 = f_rcbrt(h), r32 = r3 * r3;  // h^(-1/3), h^(-2/3)
              cf = gn2 * (r32 * r32 * r32 * r3);
            } else {
              const T hc = h * closure_cf<T>(a.fr_law, h, gn2);
              cf = T(1) / (hc * hc);
            }
            const T a1 = dt * (cf * f_sqrt(ux * ux + uy * uy));
            const T fr = f_div(T(1) + a1, T(1) + T(2) * a1);
            ux = ux * fr;
            uy = uy * fr;
          }
          if (!gt(h, hmin)) {
            ux = zero;
            uy = zero;
          }
          a.H[dst][i] = Hh;
          if constexpr (kPair) a.Hlo[dst][i] = Hl;
          a.qx[dst][i] = ux;
          a.qy[dst][i] = uy;
          if (!finite(Hh) || !finite(ux) || !finite(uy)) atomicOr(&a.ctl->status, 1);
          // negative depth: below -h_min, beyond the rounding of the FP32 bed offset in FP32-bulk
          const T negtol = kPair ? hmin + T(4) * static_cast<T>(FLT_EPSILON) * fabs(zi) : hmin;
          if (gt(-negtol, h)) atomicOr(&a.ctl->status, 2);
          if constexpr (kExtra) {
            if (trk) track_update<T, kFull>(a, i, rec, h, ux, uy, gn2, hmin, new_time(cs, 1));
          }
        }
        T u = zero, v = zero, c = zero;
        const bool wet = gt(h, hmin);
        if constexpr (SL::k64) {
          // Eq. 21's rate: a single-precision screen of every wet cell, and the exact
          // FP64 rate only where the screen comes within 1e-4 of the largest screen the
          // warp has seen for this instance (the screen is within 1e-5 of the rate, so a
          // cell below that cannot hold the instance's maximum, which stays exactly the
          // FP64 value); after the first tiles few cells pass
          const float scr = wet ? cell_rate_screen(sNx, sNy, sLn, idx, h, ux, uy, ia, a.p.g_f, a.p.cfl_mode) : 0.0f;
          smax = fmaxf(smax, __uint_as_float(__reduce_max_sync(__activemask(), __float_as_uint(scr))));
          if (wet && scr >= smax * 0.9999f) {
            cell_derived<T>(h, ux, uy, hmin, g, u, v, c);
            rrun = nmax(rrun, cell_rate<T>(sNx, sNy, sLn, idx, u, v, c, ia, a.p.cfl_mode));
          }
        } else {
          cell_derived<T>(h, ux, uy, hmin, g, u, v, c);
          if (wet) rrun = nmax(rrun, cell_rate<T>(sNx, sNy, sLn, idx, u, v, c, ia, a.p.cfl_mode));
        }
        // inflow cells: conveyance weight and depth of the new state; weir cells: the
        // weir edges' rates of Eq. 21 at the new state (h-Q edges: finalize_hq)
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int code = static_cast<int32_t>(sLR[idx[q]]) >> kLocBits;
          if (code <= kInflow) {
            const int j = kInflow - code;
            if (j < a.n_inflow) {
              a.in_pw[j] = h > hmin ? pow53(h) : zero;
              a.in_hs[j] = fmax(zero, h);
            }
          }
        }
        if constexpr (kFull) {
          if (inf.flags & 16u) {
            cell_derived<T>(h, ux, uy, hmin, g, u, v, c);
            rrun = fmax(rrun, weir_rate<T>(a, sLR, sNx, sNy, sLn, idx, Hh, Hl, zi, h, u, v, ia));
          }
          if ((inf.flags & 32u) && a.zh_n > 0) {
            // level edges: the boundary state's rate under the level of t^{n+1}
            cell_derived<T>(h, ux, uy, hmin, g, u, v, c);
            T zh_hi, zh_lo;
            level_pair<T>(a, prime ? cs.t : new_time(cs, 1), zh_hi, zh_lo);
            rrun = fmax(rrun, level_rate<T>(a, sLR, sNx, sNy, sLn, idx, zh_hi, zh_lo, zi, h, u, v, ia));
          }
        }
      }
    }

    // end of the tile: boundary flux partial (fixed order) and inflow weights -- the
    // CTA that completes the instance's last boundary / inflow tile sums the boundary
    // volume / evaluates the inflow at t^{n+1} -- then, when the CTA leaves the
    // instance, its rate max and tile count; the CTA that completes the last tile
    // advances the instance
    if (run) {
      ++cnt;
      double* scratch = reinterpret_cast<double*>(smem + L.F);  // the fluxes are consumed
      // boundary and inflow tiles: one fence and one count of both kinds (an inflow tile
      // is a boundary tile too; the counts share a 64-bit word: inflow low, boundary high)
      const bool bnd = !prime && (inf.flags & 1u);
      const bool infl = (inf.flags & 2u) != 0u;
      if (bnd || infl) {
        double bs = 0.0;
        if (bnd && !quiet) {
          // the boundary edges' l F_h (stored with the fluxes; walls 0), FP64, fixed order
          double bsum = 0.0;
          for (int k2 = tid; k2 < ne; k2 += kTile)
            if ((static_cast<int32_t>(sLR[k2]) >> kLocBits) < 0) bsum += static_cast<double>(Fs[k2]);
          bs = block_sum<kTile>(bsum, red);
        }
        if (infl && !(bnd && !quiet)) nbar<kTile>();  // every thread's inflow weights are stored
        if (tid == 0) {
          if (bnd) a.part[inf.bidx].bflux = bs;
          __threadfence();
          const unsigned long long inc = (bnd ? (1ull << 32) : 0ull) | (infl ? 1ull : 0ull);
          const unsigned long long old =
              atomicAdd(reinterpret_cast<unsigned long long*>(&a.ctl->in_done), inc);
          const bool lb = bnd && static_cast<unsigned>(old >> 32) + 1u == static_cast<unsigned>(a.n_btiles);
          const bool li = infl && static_cast<unsigned>(old) + 1u == static_cast<unsigned>(a.n_in_tiles);
          s_fin = (lb ? 1 : 0) | (li ? 2 : 0);
        }
        nbar<kTile>();
        const int fin = s_fin;
        if (fin & 1) {
          __threadfence();
          finalize_boundary<T>(a, cs, scratch);
        }
        if (fin & 2) {
          __threadfence();
          finalize_inflow<T>(a, cs, prime ? 0 : 1, red + 4, red, scratch);
        }
      }
      if (kFull && (inf.flags & 8u)) {
        // h-Q tiles: the last one's CTA evaluates the rating curve at the new stage
        __threadfence();
        nbar<kTile>();  // every thread's new state is stored
        int last_hq = 0;
        if (tid == 0)
          last_hq = atomicAdd(&a.ctl->hq_done, 1u) + 1u == static_cast<unsigned>(a.n_hq_tiles) ? 1 : 0;
        if (nbar_or<kTile>(last_hq)) {
          __threadfence();
          finalize_hq<T>(a, cs, prime ? 0 : 1, red + 4, red);
        }
      }
    }
    // the next launch's lists: a tile that was not quiet lists itself in front and the
    // tiles its halo cells lie in behind; an instance that did not step keeps its items
    // listed (nothing changed).  Where listing is not allowed, FP64 lists the tiles that
    // were not quiet, to take them first.
    const bool listed_ok = s_listed_ok != 0;
    if (!((inf.flags & kFixedFlags) != 0u || inf.item == 0) && tid == 0) {
      if (listed_ok ? (!run || !quiet) : (s_order && run && !quiet)) note(inf.item, run);
    }
    if (listed_ok && run && !quiet) {
      const int32_t* hg = reinterpret_cast<const int32_t*>(sb + RL::hidx(ne4));
      const int base = inf.item - tile;  // the instance's first item
      for (int j = tid; j < nh; j += kTile) {
        const unsigned u = static_cast<unsigned>(hg[j]) / kTile;
        if (j == 0 || static_cast<unsigned>(hg[j - 1]) / kTile != u)  // ascending: the first of each tile
          note(base + static_cast<int>(u), false);
      }
    }
    if (tid == 0) ++n_done;
    // release the tile's slot to the copy warp (each warp once it is done with it)
    __syncwarp();
    if ((tid & 31) == 0) mbar_arrive(&mb_e[k % S]);
  }
  if (cnt > 0) flush_rate();
  flush();
  // The CTA whose finished items (with the tickets its copy warp skipped) complete the
  // launch finalizes every instance that stepped and rolls the lists over (the fence
  // orders this CTA's rate maxima and list entries before its count).  A launch has at
  // least one ticket (item 0 is fixed), so some CTA completes it.
  int last = 0;
  if (tid == 0) {
    const int total = n_done + s_skip;
    if (total > 0) {
      __threadfence();
      const unsigned long long inc = (static_cast<unsigned long long>(n_done) << 32) | static_cast<unsigned>(total);
      const unsigned long long old = atomicAdd(reinterpret_cast<unsigned long long*>(&sched[10]), inc);
      last = static_cast<int>(old & 0xffffffffull) + total == s_tickets ? 1 : 0;
    }
  }
  if (nbar_or<kTile>(last)) {
    __threadfence();
    const int roll_tid = min(((g.n_inst + 31) / 32) * 32, kTile - 32);  // a warp with no instance (if any)
    for (int k = tid; k < g.n_inst; k += kTile) {
      // (the fields finalize_step reads plainly are not written during a launch)
      const PipeItem& it = items[g.inst_item[k]];
      const Ctl& cs = *it.ctl;
      if (prime || cs.active) finalize_step<T>(*static_cast<const InstDesc<T>*>(it.desc), cs, prime ? 0 : 1);
    }
    // launch stamps restart before they overflow: the marks forget every listing and
    // the next launch takes every item
    const int stamp = s_stamp;
    const bool wrap = stamp + 1 >= kStampMax;
    if (wrap)
      for (int j = tid; j < 2 * n_items; j += kTile)
        if (__ldcg(&mark[j]) != kFixedMark) mark[j] = -1;
    if (wrap) nbar<kTile>();
    if (tid == roll_tid) {
      // every other CTA has finished with the counters (its count came before this one)
      volatile int* vs = sched;
      const int nf = vs[3], nb = vs[6], ok = vs[9], done = vs[11];
      // a list that holds most items: the next launch takes them all in work-list order
      // (and without lists built in this launch, so does the next); after a prime pass,
      // every item in work-list order, building the lists
      const bool dense = 4LL * (nf + nb) > 3LL * (n_items - g.n_fixed) || (ok && !s_listed_ok);
      const int next_mode = !ok ? 0 : (prime ? 3 : (dense ? 2 : 1));
      vs[3] = 0;
      vs[6] = 0;
      vs[10] = 0;
      vs[11] = 0;
      vs[12] = done;
      vs[4] = wrap ? 0 : nf;
      vs[7] = wrap ? 0 : nb;
      vs[8] = wrap ? 0 : next_mode;
      vs[2] = wrap ? 0 : stamp + 1;
      __threadfence();
    }
  }
}

}  // namespace bm
