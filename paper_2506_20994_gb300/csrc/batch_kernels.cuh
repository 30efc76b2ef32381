// The batched operator's kernels (batch.cu): one persistent kernel per dtype
// for the whole batch, whatever the polynomial orders in it.
//
// Each CTA (kBatchThreads threads) walks its own list of groups; a group is
// a run of work items (element ranges of meshes) that share one lx and one
// thread layout, and the CTA runs the matching device body over it:
//  * fp64, lx in {6, 8, 10} with centro-antisymmetric matrices: the
//    persistent even-odd body of the operator handle (ax_eo_persist.cuh).
//    The CTA splits into kBatchThreads / NTB independent slots of NTB
//    threads, each with its own shared memory, bulk-copy barrier and named
//    barrier; slot q takes elements q, q + S, ... of the group's
//    concatenated items and streams the next one's geometry in while it
//    computes the current one.  The arithmetic is the handle's, so results
//    equal ax_op_apply's bit for bit.
//  * fp32, lx in {6, 8, 10} with 16-byte aligned arrays: the persistent
//    even-odd fp32 body of ax_helm_f32 (ax_eo32.cuh), in slots the same way;
//  * every other case: the k-loop body of the single-mesh kernels
//    (double-float for fp64, fp32 for fp32) in chunks of
//    kBatchThreads / lx^2 elements, bit for bit ax_helm's / ax_helm_f32's.
// Groups are separated by a block barrier (the shared memory changes role).
// No atomics and no waits between CTAs.  CTAs of 256 threads, several per SM,
// so that one CTA's block barriers (k-loop bodies) leave the others running
// (measured: one 512-thread CTA per SM was 14-22 % slower on the uneven
// benchmark batch).
#pragma once

#include "ax_df64.cuh"
#include "ax_eo32.cuh"
#include "ax_eo_persist.cuh"
#include "ax_kstep.cuh"

namespace ax {

constexpr int kBatchThreads = 256;

struct BatchMeshDev {
  int lx;
  void *w;
  const void *u, *dx, *dxt, *h1, *g[6];
};

struct BatchItem {
  int mesh, nel;
  long long e0;
};

// A group: items [ib, ie) of one body key (2 lx + layout).
struct BatchGroup {
  int key, ib, ie;
};

// Thread layout of a group.
enum BatchBody : int { kBodyKLoop = 0, kBodyEvenOdd = 1 };

// Orders whose even-odd body fits a batch CTA (lx 12 needs 432 threads).
__host__ __device__ constexpr bool batch_eo_ok(int lx) { return lx == 6 || lx == 8 || lx == 10; }

// Elements per chunk of the k-loop body in a batch CTA.
__host__ __device__ constexpr int batch_kloop_epb(int lx) {
  return kBatchThreads / (lx * lx) < 1 ? 1 : kBatchThreads / (lx * lx);
}

// The even-odd slots' sequence: elements slot, slot + S, ... of the
// concatenation of items [ib, ie); M: the body's mesh operands.
template <class M>
struct SeqItemsT {
  static constexpr bool kRotate10 = false;  // line layout of the fp64 body, see eop::lpos
  const BatchItem *items;
  int ib, ie, slot, S;
  const M *meshes;
  AX_D bool norm(eop::EopPos &p) const {
    while (p.it < ie && p.off >= items[p.it].nel) {
      p.off -= items[p.it].nel;
      ++p.it;
    }
    return p.it < ie;
  }
  AX_D bool first(eop::EopPos &p) const {
    p = eop::EopPos{ib, (long long)slot};
    return norm(p);
  }
  AX_D bool advance(const eop::EopPos &p, eop::EopPos &q) const {
    q = eop::EopPos{p.it, p.off + S};
    return norm(q);
  }
  AX_D int mesh_of(const eop::EopPos &p) const { return items[p.it].mesh; }
  AX_D long long elem(const eop::EopPos &p) const { return items[p.it].e0 + p.off; }
  AX_D const M &mesh(int m) const { return meshes[m]; }
};
using SeqItems = SeqItemsT<eop::EopMesh>;
using F32Mesh = e32::Mesh<float, float>;

// Bytes of one even-odd slot's shared memory (128-byte aligned).
template <int LX>
constexpr size_t batch_eo_slot_bytes() {
  return (eop::Cfg<LX>::SMEM + 127) / 128 * 128;
}
template <int LX>
constexpr int batch_eo_slots() {
  return kBatchThreads / eop::Cfg<LX>::NTB;
}

template <int LX>
__device__ __noinline__ void batch_run_eo(const BatchGroup &G, const BatchItem *items,
                                             const eop::EopMesh *emesh, unsigned char *sm,
                                             int *err) {
  using C = eop::Cfg<LX>;
  constexpr int S = batch_eo_slots<LX>();
  const int slot = (int)threadIdx.x / C::NTB;
  if (slot >= S) return;  // threads beyond the last whole slot sit the group out
  const int tid = (int)threadIdx.x - slot * C::NTB;
  const unsigned bid = 1u + (unsigned)slot;
  const SeqItems seq{items, G.ib, G.ie, slot, S, emesh};
  auto sync = [bid] { asm volatile("bar.sync %0, %1;" ::"r"(bid), "r"(C::NTB) : "memory"); };
  auto sync_and = [bid](bool p) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred a, b;\n\tsetp.ne.u32 a, %1, 0;\n\t"
        "bar.red.and.pred b, %2, %3, a;\n\tselp.u32 %0, 1, 0, b;\n\t}"
        : "=r"(r)
        : "r"((unsigned)p), "r"(bid), "r"(C::NTB)
        : "memory");
    return r != 0u;
  };
  double dsum = 0.0;
  const eop::EopUpd up{nullptr, nullptr, nullptr, nullptr, 0.0, false};
  eop::eop_run<LX, false, false>(sm + (size_t)slot * batch_eo_slot_bytes<LX>(), tid, seq, sync,
                                 sync_and, err, up, dsum);
}

// fp32 meshes of these orders with 16-byte aligned arrays run the even-odd
// fp32 body (that of ax_helm_f32, bit for bit); its lx = 12 form needs 432
// threads, so lx 12 runs the k-loop body here.
__host__ __device__ constexpr bool batch_e32_ok(int lx) { return lx == 6 || lx == 8 || lx == 10; }
template <int LX>
constexpr size_t batch_e32_slot_bytes() {
  return (e32::Cfg<LX, float, float>::SMEM + 127) / 128 * 128;
}
template <int LX>
constexpr int batch_e32_slots() {
  return kBatchThreads / e32::Cfg<LX, float, float>::NTB;
}

template <int LX>
__device__ __noinline__ void batch_run_e32(const BatchGroup &G, const BatchItem *items,
                                           const F32Mesh *fmesh, unsigned char *sm, int *err) {
  using C = e32::Cfg<LX, float, float>;
  constexpr int S = batch_e32_slots<LX>();
  const int slot = (int)threadIdx.x / C::NTB;
  if (slot >= S) return;
  const int tid = (int)threadIdx.x - slot * C::NTB;
  const unsigned bid = 1u + (unsigned)slot;
  const SeqItemsT<F32Mesh> seq{items, G.ib, G.ie, slot, S, fmesh};
  auto sync = [bid] { asm volatile("bar.sync %0, %1;" ::"r"(bid), "r"(C::NTB) : "memory"); };
  auto sync_and = [bid](bool p) {
    unsigned r;
    asm volatile(
        "{\n\t.reg .pred a, b;\n\tsetp.ne.u32 a, %1, 0;\n\t"
        "bar.red.and.pred b, %2, %3, a;\n\tselp.u32 %0, 1, 0, b;\n\t}"
        : "=r"(r)
        : "r"((unsigned)p), "r"(bid), "r"(C::NTB)
        : "memory");
    return r != 0u;
  };
  double dsum = 0.0;
  e32::e32_run<LX, float, float, false, false, false>(sm + (size_t)slot * batch_e32_slot_bytes<LX>(),
                                               tid, seq, sync, sync_and, err, dsum);
}

template <bool F64, int LX>
__device__ __noinline__ void batch_run_kloop(const BatchGroup &G, const BatchItem *items,
                                                const BatchMeshDev *meshes, unsigned char *sm) {
  constexpr int EPB = batch_kloop_epb(LX);
  for (int it = G.ib; it < G.ie; ++it) {
    const BatchItem itm = items[it];
    const BatchMeshDev m = meshes[itm.mesh];
    for (int q = 0; q < itm.nel; q += EPB) {
      const int nel = itm.nel - q < EPB ? itm.nel - q : EPB;
      if constexpr (F64) {
        df64_body<LX>((double *)m.w, (const double *)m.u, (const double *)m.dx,
                      (const double *)m.dxt, (const double *)m.h1, (const double *)m.g[0],
                      (const double *)m.g[1], (const double *)m.g[2], (const double *)m.g[3],
                      (const double *)m.g[4], (const double *)m.g[5], itm.e0 + q, nel, EPB, sm);
      } else {
        kstep_body<LX, float, float, float, float, true, false, kstep_vec<LX, float>()>(
            (float *)m.w, (const float *)m.u, (const float *)m.dx, (const float *)m.dxt,
            (const float *)m.h1, (const float *)m.g[0], (const float *)m.g[1],
            (const float *)m.g[2], (const float *)m.g[3], (const float *)m.g[4],
            (const float *)m.g[5], itm.e0 + q, nel, EPB, sm);
      }
      __syncthreads();  // the next chunk reuses the shared memory
    }
  }
}

// Per-dtype host helpers, defined in batch_f64.cu / batch_f32.cu: one
// persistent launch of the dtype's kernel; the shared-memory bytes a group
// of key (2 lx + layout) needs; the resident CTAs per SM at `smem` bytes
// (raising the kernel's shared-memory limit first).
int batch_launch_f64(int nblocks, size_t smem, const BatchMeshDev *meshes,
                     const eop::EopMesh *emesh, const BatchItem *items, const BatchGroup *groups,
                     const int *cta_start, int *err, cudaStream_t st);
int batch_launch_f32(int nblocks, size_t smem, const BatchMeshDev *meshes,
                     const F32Mesh *fmesh, const BatchItem *items, const BatchGroup *groups,
                     const int *cta_start, int *err, cudaStream_t st);
size_t batch_key_smem_f64(int key);
size_t batch_key_smem_f32(int key);
int batch_setup_f64(size_t smem, int *blocks_per_sm);
int batch_setup_f32(size_t smem, int *blocks_per_sm);

}  // namespace ax
