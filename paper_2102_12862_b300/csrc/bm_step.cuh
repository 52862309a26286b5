// bm_step.cuh -- the fused step kernel (sm_103a): persistent CTAs of eight compute
// warps and one copy warp, a shared-memory pipeline fed by bulk asynchronous copies.
//
// Each CTA walks the launch's work items (tiles of 256 Hilbert-ordered cells of some
// instance) with a stride of gridDim.x.  Its copy warp streams every tile's data into
// shared memory ahead of the compute warps, in two groups completed on mbarriers:
//   group A  bulk copies (cp.async.bulk) of the tile record (inverse areas, slots,
//            edge codes and geometry, halo list), the instance descriptor and a
//            snapshot of the instance's control block;
//   group B  issued once A has landed (its addresses come from A): bulk copies of the
//            tile's slices of the state arrays (surface, discharge, bed, g n^2, FP64:
//            velocity and celerity) and cp.async gathers of the halo cells' values
//            (other tiles' cells, in ascending index order).
// Three A slots and two B slots; the compute warps release a tile's slots when they
// are done with it (empty barriers) and the copy warp refills them, so copying never
// stalls the arithmetic.  The compute warps read shared memory only (BASEMENT v3,
// Section "Numerical solution"):
//   phase D  wet/dry flag of every local cell (FP32-bulk: also its velocity/celerity);
//            a tile whose cells and halo are dry, at rest and without inflow is quiet;
//   phase F  each tile edge once: modified states on max(z_L, z_R), HLLC flux in the
//            edge frame, pre-balanced pressure, wall / transmissive / inflow states;
//            an edge whose two cells are dry, or whose modified depths are both zero,
//            contributes exactly zero and is not evaluated;
//   phase I  each cell gathers its three edge contributions (Eq. 12), split Manning
//            friction (Eq. 2, Table 1), U^{n+1} to HBM, the lambda/rho rate of Eq. 21;
//            a dry cell at rest with three skipped edges (every cell of a quiet tile)
//            is copied through unchanged;
//   flush    when the CTA leaves an instance: max rate and tile count to the
//            instance's control block; the CTA that completes an instance finalizes it
//            (next dt, time, boundary volume, inflow split) -- no second launch.
// Every mbarrier wait is bounded (about a second): on timeout the CTA flags the
// instance (status bit 2), its copy warp drains what it issued, and all warps return.
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
// the instruction meanwhile (suspend-time hint 0.1 ms).
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(saddr(b)), "r"(parity), "r"(100000u)
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

// Order-preserving integer key of a double (for x, y not NaN: key(x) <= key(y)
// implies x <= y), so wet/dry tests of FP64 cells need no FP64 instruction.
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
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
  int next_inst;  // instance of the CTA's next tile (-1: none)
  int pad[2];
};

constexpr int kASlots = 3, kBSlots = 2;

template <typename T>
struct StepLayout {
  static constexpr bool k64 = sizeof(T) == 8;
  static constexpr int S = sizeof(T);
  static constexpr int kNA = k64 ? 7 : 5;  // staged per-cell arrays
  // array order: FP64 H qx qy z u v c; FP32-bulk H Hlo qx qy z
  static constexpr int kH = 0, kHl = 1, kQx = k64 ? 1 : 2, kQy = k64 ? 2 : 3, kZ = k64 ? 3 : 4, kU = 4, kV = 5, kC = 6;
  static constexpr uint32_t kDesc = (sizeof(InstDesc<T>) + 15) & ~15u;
  uint32_t ne4, nh4, nloc;
  uint32_t desc, ctl, info, aslot;  // within an A slot (record at 0), A slot size
  uint32_t gn2, bslot, b0;          // within a B slot (arrays at 0), B slot size, first B slot
  uint32_t F, uvc, dry, skip, red, total;  // from the start of shared memory
  BM_HD StepLayout(uint32_t ne4_, uint32_t nh4_) {
    ne4 = ne4_;
    nh4 = nh4_;
    nloc = kTile + nh4;
    desc = align16(RecLayout<S>::bytes(ne4, nh4));
    ctl = desc + kDesc;
    info = ctl + static_cast<uint32_t>(sizeof(Ctl));
    aslot = (info + static_cast<uint32_t>(sizeof(StageInfo)) + 127u) & ~127u;
    gn2 = kNA * nloc * S;
    bslot = (gn2 + kTile * S + 127u) & ~127u;
    b0 = kASlots * aslot;
    F = b0 + kBSlots * bslot;
    uvc = F + 5 * ne4 * S;
    dry = uvc + (k64 ? 0u : 3 * nloc * S);
    skip = dry + align16(nloc);
    red = skip + align16(ne4);
    total = red + 10 * 8;
  }
};

// ------------------------------------------------------------------ the copy warp

// Group A of a tile into an A slot (all lanes of the copy warp).
template <typename T>
__device__ __forceinline__ void issue_a(const StepLayout<T>& L, unsigned char* sa, const PipeItem& it, int next_inst,
                                        uint64_t* mb, int lane) {
  if (lane == 0) {
    StageInfo* inf = reinterpret_cast<StageInfo*>(sa + L.info);
    inf->tile = it.tile;
    inf->ne = static_cast<int>(it.ne_nh & 0xffffu);
    inf->nh = static_cast<int>(it.ne_nh >> 16);
    inf->inst = it.inst;
    inf->flags = it.flags;
    inf->next_inst = next_inst;
    // the arrival (release) orders the stores above before the phase completes
    mbar_expect_tx(mb, it.rec_bytes + StepLayout<T>::kDesc + static_cast<uint32_t>(sizeof(Ctl)));
  }
  __syncwarp();
  if (lane == 0)
    bulk_g2s(sa, it.rec, it.rec_bytes, mb);
  else if (lane == 1)
    bulk_g2s(sa + L.desc, it.desc, StepLayout<T>::kDesc, mb);
  else if (lane == 2)
    bulk_g2s(sa + L.ctl, it.ctl, static_cast<uint32_t>(sizeof(Ctl)), mb);
}

// Group B of a tile into a B slot, from its landed A slot (all lanes of the copy warp):
// state slices by bulk copy (lane j < kNA: array j, lane kNA: g n^2), halo values by
// cp.async, each lane arriving on mb when its gathers have landed.
template <typename T>
__device__ __forceinline__ void issue_b(const StepLayout<T>& L, const unsigned char* sa, unsigned char* sbb,
                                        uint64_t* mb, int lane) {
  using SL = StepLayout<T>;
  const StageInfo& inf = *reinterpret_cast<const StageInfo*>(sa + L.info);
  const InstDesc<T>& a = *reinterpret_cast<const InstDesc<T>*>(sa + L.desc);
  const int par = reinterpret_cast<const Ctl*>(sa + L.ctl)->parity;
  const T* src[SL::kNA];
  if constexpr (SL::k64) {
    src[0] = a.H[par]; src[1] = a.qx[par]; src[2] = a.qy[par]; src[3] = a.z;
    src[4] = a.u[par]; src[5] = a.v[par]; src[6] = a.c[par];
  } else {
    src[0] = a.H[par]; src[1] = a.Hlo[par]; src[2] = a.qx[par]; src[3] = a.qy[par]; src[4] = a.z;
  }
  T* arr = reinterpret_cast<T*>(sbb);
  constexpr uint32_t kSlice = kTile * sizeof(T);
  if (lane == 0) mbar_expect_tx(mb, (SL::kNA + 1) * kSlice);
  __syncwarp();
  const T* sj = a.gn2;
  unsigned char* dj = sbb + L.gn2;
#pragma unroll
  for (int j = 0; j < SL::kNA; ++j)
    if (lane == j) {
      sj = src[j];
      dj = reinterpret_cast<unsigned char*>(arr + j * L.nloc);
    }
  if (lane <= SL::kNA) bulk_g2s(dj, sj + static_cast<size_t>(inf.tile) * kTile, kSlice, mb);
  const int32_t* hidx = reinterpret_cast<const int32_t*>(sa + RecLayout<SL::S>::hidx(round4(inf.ne)));
  for (int h = lane; h < inf.nh; h += 32) {
    const int gi = hidx[h];
#pragma unroll
    for (int j = 0; j < SL::kNA; ++j) cp_async<sizeof(T)>(arr + j * L.nloc + kTile + h, src[j] + gi);
  }
  cp_async_arrive(mb);
}

// ------------------------------------------------------------------ the step

template <typename T>
constexpr int kMinBlocks = sizeof(T) == 8 ? 2 : 3;

// One step (prime = 0) or prime pass (prime = 1: no update; derived data, inflow
// weights and the dt of the current state) over a work list.  ne4max / nh4max: the
// largest record of the list (they fix the shared-memory layout).  A single state is
// a list of one instance's tiles, so a run executes the same machine code alone and in
// a batch and gives bitwise the same result.
template <typename T>
__global__ void __launch_bounds__(kStepThreads, kMinBlocks<T>) step_pipe(const PipeItem* __restrict__ items,
                                                                         int n_items, int ne4max, int nh4max,
                                                                         int prime) {
  using SL = StepLayout<T>;
  using RL = RecLayout<SL::S>;
  constexpr bool kPair = !SL::k64;
  extern __shared__ __align__(128) unsigned char smem[];
  // full / empty barriers of the A slots and the B slots
  __shared__ __align__(8) uint64_t mb_fa[kASlots], mb_ea[kASlots], mb_fb[kBSlots], mb_eb[kBSlots];
  __shared__ int s_abort;
  const SL L(static_cast<uint32_t>(ne4max), static_cast<uint32_t>(nh4max));
  const int tid = threadIdx.x;
  const int G = gridDim.x;
  if (static_cast<int>(blockIdx.x) >= n_items) return;
  auto aslot = [&](int k) { return smem + (k % kASlots) * L.aslot; };
  auto bslot = [&](int k) { return smem + L.b0 + (k & 1) * L.bslot; };
  const int n_mine = (n_items - static_cast<int>(blockIdx.x) + G - 1) / G;  // this CTA's tiles

  if (tid == 0) {
    for (int s = 0; s < kASlots; ++s) {
      mbar_init(&mb_fa[s], 1);
      mbar_init(&mb_ea[s], kTile / 32);
    }
    for (int s = 0; s < kBSlots; ++s) {
      mbar_init(&mb_fb[s], 1 + 32);
      mbar_init(&mb_eb[s], kTile / 32);
    }
    mbar_init_fence();
    s_abort = 0;
  }
  __syncthreads();

  if (tid >= kTile) {
    // ---------------------------------------------------------------- copy warp
    const int lane = tid - kTile;
    volatile int* abort_flag = &s_abort;
    // work items are read one tile ahead of their use, so no copy waits on that read
    auto item = [&](int j) -> PipeItem { return j < n_mine ? items[blockIdx.x + j * G] : PipeItem{}; };
    int a_next = 0;  // next tile whose group A is issued
    bool ok = true;
    PipeItem it0 = item(0), it1 = item(1), it2 = item(2);
    issue_a<T>(L, aslot(0), it0, n_mine > 1 ? it1.inst : -1, &mb_fa[0], lane);
    a_next = 1;
    if (n_mine > 1) {
      issue_a<T>(L, aslot(1), it1, n_mine > 2 ? it2.inst : -1, &mb_fa[1], lane);
      a_next = 2;
    }
    PipeItem ia = it2, ib = item(3);  // tiles k+2 and k+3 at iteration k
    for (int k = 0; k < n_mine && ok; ++k) {
      // B(k): its A landed and tile k-2 released its B slot
      if (k >= 2) ok = mbar_wait(&mb_eb[k & 1], ((k - 2) >> 1) & 1);
      ok = ok && mbar_wait(&mb_fa[k % kASlots], (k / kASlots) & 1);
      ok = __all_sync(0xffffffffu, ok) && !*abort_flag;
      if (!ok) break;
      issue_b<T>(L, aslot(k), bslot(k), &mb_fb[k & 1], lane);
      // A(k+2): tile k-1 released its A slot
      if (k + 2 < n_mine) {
        if (k >= 1) ok = mbar_wait(&mb_ea[(k + 2) % kASlots], ((k - 1) / kASlots) & 1);
        ok = __all_sync(0xffffffffu, ok) && !*abort_flag;
        if (!ok) break;
        issue_a<T>(L, aslot(k + 2), ia, k + 3 < n_mine ? ib.inst : -1, &mb_fa[(k + 2) % kASlots], lane);
        a_next = k + 3;
        ia = ib;
        ib = item(k + 4);
      }
    }
    cp_async_wait_all();
    if (!ok) {
      if (lane == 0) {
        *abort_flag = 1;
        atomicOr(&items[blockIdx.x].ctl->status, 4);
      }
      // let the bulk copies of the last groups issued land before the CTA exits
      for (int j = a_next - 1; j >= 0 && j >= a_next - kASlots; --j) (void)mbar_wait(&mb_fa[j % kASlots], (j / kASlots) & 1);
    }
    return;
  }

  // ------------------------------------------------------------------ compute warps
  T* Fs = reinterpret_cast<T*>(smem + L.F);
  unsigned char* dry = smem + L.dry;
  unsigned char* skip = smem + L.skip;
  double* red = reinterpret_cast<double*>(smem + L.red);
  const T zero = T(0);
  volatile int* abort_flag = &s_abort;
  double rrun = 0.0;  // this CTA's max Eq. 21 rate over the current instance's tiles
  unsigned cnt = 0;   // tiles of the current instance this CTA completed
  int w = blockIdx.x;
  for (int k = 0; k < n_mine; ++k) {
    unsigned char* sb = aslot(k);
    unsigned char* bs_ = bslot(k);
    {
      const bool ok = mbar_wait(&mb_fa[k % kASlots], (k / kASlots) & 1) && mbar_wait(&mb_fb[k & 1], (k >> 1) & 1);
      if (nbar_or<kTile>(!ok || *abort_flag)) {
        if (tid == 0) {
          *abort_flag = 1;
          atomicOr(&items[w].ctl->status, 4);
        }
        return;
      }
    }

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
    const T* arr = reinterpret_cast<const T*>(bs_);
    const T* sH = arr + SL::kH * L.nloc;
    const T* sHl = arr + SL::kHl * L.nloc;  // FP32-bulk only
    const T* sQx = arr + SL::kQx * L.nloc;
    const T* sQy = arr + SL::kQy * L.nloc;
    const T* sZ = arr + SL::kZ * L.nloc;
    const T* sGn2 = reinterpret_cast<const T*>(bs_ + L.gn2);
    T* U;
    T* V;
    T* C;
    if constexpr (SL::k64) {
      U = const_cast<T*>(arr + SL::kU * L.nloc);
      V = const_cast<T*>(arr + SL::kV * L.nloc);
      C = const_cast<T*>(arr + SL::kC * L.nloc);
    } else {
      U = reinterpret_cast<T*>(smem + L.uvc);
      V = U + L.nloc;
      C = V + L.nloc;
    }
    const bool run = prime || cs.active;
    T dt, quni, g, hg, hmin;
    step_consts(&cs, a.p, dt, quni, g, hg, hmin);
    const double qscale = cs.qscale;
    const int wpos = cs.wpos;
    const int par = cs.parity;

    // phase D: wet/dry flags (FP32-bulk: velocity and celerity) of tile and halo cells.
    // A tile whose cells and halo cells are all dry, whose cells are at rest and which
    // has no inflow edge is quiet: every flux is zero and U^{n+1} = U^n.
    bool tq = true;
    if (run) {
      for (int j = tid; j < kTile + nh; j += kTile) {
        const T Hj = sH[j], Hlj = kPair ? sHl[j] : zero, zj = sZ[j];
        const bool dj = cell_dry(Hj, Hlj, zj);
        dry[j] = dj ? 1 : 0;
        tq = tq && dj && (j >= kTile || (is_zero(sQx[j]) && is_zero(sQy[j])));
        if constexpr (kPair) {
          T u = zero, v = zero, c = zero;  // dry: at rest, zero celerity
          if (!dj) cell_derived<T>(depth_of(Hj, Hlj, zj), sQx[j], sQy[j], hmin, g, u, v, c);
          U[j] = u;
          V[j] = v;
          C[j] = c;
        }
      }
    }
    const bool quiet = nbar_and<kTile>(tq) && !prime && !(inf.flags & 2u);

    // phase F: edges
    double bsum = 0.0;
    if (run && !prime && !quiet) {
      for (int k2 = tid; k2 < ne; k2 += kTile) {
        const uint32_t lr = sLR[k2];
        const int lL = static_cast<int>(lr & (kMaxLocal - 1));
        const int R = static_cast<int32_t>(lr) >> kLocBits;
        const int lR = R >= 0 ? R : lL;
        const bool inflow = R <= kInflow;
        T f0 = zero, f1 = zero, f2 = zero, f3 = zero, f4 = zero;
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
          const T zs = fmax(zL, zR);
          const T h1 = fmax(zero, depth_of(HLh, HLl, zs));
          const T h2 = fmax(zero, depth_of(HRh, HRl, zs));
          if (h1 > zero || h2 > zero || inflow) {
            skipped = 0;
            const T nx = sNx[k2], ny = sNy[k2], l = sLn[k2];
            const T uL = U[lL], vL = V[lL], cL = C[lL];
            const T unL = uL * nx + vL * ny, utL = -uL * ny + vL * nx;
            T un2, ut2, c1, c2;
            if (R >= 0) {
              const T uR = U[lR], vR = V[lR], cR = C[lR];
              // the side with the higher bed keeps its own depth, hence its own celerity
              const bool lhi = zL >= zR;
              const T clo = f_sqrt(g * (lhi ? h2 : h1));
              c1 = lhi ? cL : clo;
              c2 = lhi ? clo : cR;
              un2 = uR * nx + vR * ny;
              ut2 = -uR * ny + vR * nx;
            } else {
              c1 = cL;
              c2 = cL;
              un2 = (R == kWall) ? -unL : unL;  // wall: mirrored normal velocity
              ut2 = utL;
            }
            T F0, F1, F2, pL, pR;
            hllc<T>(h1, unL, utL, c1, h2, un2, ut2, c2, hg, F0, F1, F2, pL, pR);
            T GL = F1 - pL;
            const T GR = F1 - pR;
            if (R == kWall) {
              F0 = zero;  // impermeable, frictionless
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
            if (R < 0) bsum += static_cast<double>(l * F0);
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
      }
    }
    nbar<kTile>();

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
      if (quiet ||
          (!prime && skip[idx[0]] && skip[idx[1]] && skip[idx[2]] && dry[tid] && is_zero(qxi) && is_zero(qyi))) {
        // no flux, dry and at rest: U^{n+1} = U^n, velocity and celerity zero
        a.H[dst][i] = Hh;
        if constexpr (kPair) a.Hlo[dst][i] = Hl;
        a.qx[dst][i] = zero;
        a.qy[dst][i] = zero;
        if constexpr (SL::k64) {
          a.u[dst][i] = zero;
          a.v[dst][i] = zero;
          a.c[dst][i] = zero;
        }
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int code = static_cast<int32_t>(sLR[idx[q]]) >> kLocBits;
          if (code <= kInflow) {
            a.in_pw[kInflow - code] = zero;
            a.in_hs[kInflow - code] = zero;
          }
        }
      } else {
        T h = depth_of(Hh, Hl, zi), ux = qxi, uy = qyi;
        if (!prime) {
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
          h = depth_of(Hh, Hl, zi);
          if (h > hmin && gn2 > zero) {
            // split friction: two semi-implicit stages, Heun average
            const T cf = f_div(gn2, h * h * f_cbrt(h));
            const T k0 = cf * f_sqrt(ux * ux + uy * uy);
            const T d0 = f_div(T(1), T(1) + dt * k0);
            const T q1x = ux * d0, q1y = uy * d0;
            const T k1 = cf * f_sqrt(q1x * q1x + q1y * q1y);
            const T d1 = f_div(T(1), T(1) + dt * k1);
            ux = T(0.5) * (ux + q1x * d1);
            uy = T(0.5) * (uy + q1y * d1);
          }
          if (!(h > hmin)) {
            ux = zero;
            uy = zero;
          }
          a.H[dst][i] = Hh;
          if constexpr (kPair) a.Hlo[dst][i] = Hl;
          a.qx[dst][i] = ux;
          a.qy[dst][i] = uy;
          if (!isfinite(Hh) || !isfinite(ux) || !isfinite(uy)) atomicOr(&a.ctl->status, 1);
          // negative depth: below -h_min, beyond the rounding of the FP32 bed offset in FP32-bulk
          const T negtol = kPair ? hmin + T(4) * static_cast<T>(FLT_EPSILON) * fabs(zi) : hmin;
          if (h < -negtol) atomicOr(&a.ctl->status, 2);
        }
        const int out = prime ? par : dst;
        T u, v, c;
        cell_derived<T>(h, ux, uy, hmin, g, u, v, c);
        if constexpr (SL::k64) {
          a.u[out][i] = u;
          a.v[out][i] = v;
          a.c[out][i] = c;
        }
        if (h > hmin) rrun = fmax(rrun, static_cast<double>(cell_rate<T>(sNx, sNy, sLn, idx, u, v, c, ia, a.p.cfl_mode)));
        // inflow cells: conveyance weight and depth of the new state
#pragma unroll
        for (int q = 0; q < 3; ++q) {
          const int code = static_cast<int32_t>(sLR[idx[q]]) >> kLocBits;
          if (code <= kInflow) {
            a.in_pw[kInflow - code] = h > hmin ? pow53(h) : zero;
            a.in_hs[kInflow - code] = fmax(zero, h);
          }
        }
      }
    }

    // end of the tile: boundary flux partial (fixed order), then, when the CTA leaves
    // the instance, its rate max and tile count; the last CTA finalizes the instance
    if (run) {
      ++cnt;
      if (!prime && (inf.flags & 1u)) {
        const double bs = quiet ? 0.0 : block_sum<kTile>(bsum, red);
        if (tid == 0) a.part[tile].bflux = bs;
      }
    }
    const bool leave = inf.next_inst != inf.inst;
    if (leave && cnt > 0) {
      const double r = block_max<kTile, double>(rrun, red);
      int is_last = 0;
      if (tid == 0) {
        if (r > 0.0) atomicMax(&a.ctl->rmax_bits, static_cast<unsigned long long>(__double_as_longlong(r)));
        __threadfence();
        const unsigned prev = atomicAdd(&a.ctl->done, cnt);
        is_last = (prev + cnt == static_cast<unsigned>(a.n_tiles)) ? 1 : 0;
      }
      if (nbar_or<kTile>(is_last)) {
        __threadfence();
        finalize_instance<T>(a, prime ? 0 : 1, red, red + 8);
      }
      rrun = 0.0;
      cnt = 0;
    }
    // release the tile's slots to the copy warp (each warp once it is done with them)
    __syncwarp();
    if ((tid & 31) == 0) {
      mbar_arrive(&mb_ea[k % kASlots]);
      mbar_arrive(&mb_eb[k & 1]);
    }
    w += G;

  }
}

}  // namespace bm
