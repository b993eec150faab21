// Matrix-free operator applies and exact operator diagonals.
//
// One thread per leaf element, elements in Morton order so that neighbouring threads share most
// of their nodes in cache. Each thread gathers its 8 corner values (hanging corners interpolated
// from their parents), applies the element operator with 2x2x2 Gauss quadrature and geometry
// recomputed from the octant level, and scatter-adds the result (hanging corners distributed
// back to their parents), i.e. y = P^T (sum_e A_e) P x without storing any matrix.
#include "ops.cuh"
#include "reduce.cuh"

namespace chns {

constexpr int kApplyThreads = 128;

// Coefficient fields the patch kernels gather into shared memory (none for operators that
// ignore them).
template <class K>
constexpr int gathered_fields() {
  return IgnoresFields<K>::value ? 0 : K::NF;
}

template <class K, class T, class S, class C>
__global__ void __launch_bounds__(kApplyThreads) k_apply(MeshDev m, DevParams p, CoefArgs<C> cf,
                                                         const S* __restrict__ x, S* __restrict__ y) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_elem) return;
  int idx[8];
  load_corners(m, e, idx);
  const Geo<T> g = geometry<T>(m, e);
  K k;
  k.load(m, p, cf, idx, g);
  T xin[K::NC][8];
#pragma unroll
  for (int c = 0; c < K::NC; ++c) gather<T, K::DIR>(m, idx, x + c * m.n_nodes, xin[c]);
  T r[K::NC][8];
  k.apply(g, p, xin, r);
#pragma unroll
  for (int c = 0; c < K::NC; ++c) scatter<T, K::DIR>(m, idx, r[c], y + c * m.n_nodes);
}

// Patch apply: one CTA per patch (kPatchElems Morton-consecutive elements, one thread each).
//  1. the patch's regular slots are gathered once into shared memory (input components and
//     coefficient fields), Dirichlet nodes as zero for DIR operators;
//  2. hanging slots are interpolated there from their parent slots (mean of 2 or 4);
//  3. each thread applies its element operator reading its 8 corners from shared memory and adds
//     the result into shared accumulators (shared-memory atomics);
//  4. hanging accumulators are distributed to their parents with the same weights;
//  5. each regular slot is written once: a plain store when the patch owns the node, a global
//     atomic add otherwise (nodes on the patch boundary). y must be zero on entry.
// With PQ the block sums of the element energies x_e . A_e x_e (summing to x^T A x) are added to
// S_cg[kCgPq0 + par] with an FP64 atomic; operators with ENERGY form them from their quadrature
// data (non-negative terms), the others as x_e . (A_e x_e) in double-float.
template <class K, class T, class S, class C, bool PQ, bool CGP>
__global__ void __launch_bounds__(kPatchElems, K::MIN_CTAS)
k_apply_patch(MeshDev m, DevParams p, CoefArgs<C> cf, const S* __restrict__ x, S* __restrict__ y,
              double* __restrict__ S_cg, int par, int fcg, const S* __restrict__ zcg,
              S* __restrict__ pout) {
  constexpr int NC = K::NC, NF = gathered_fields<K>();
  // shared accumulators: the arithmetic type, or FP64 for double-float (same size)
  using U = AccumT<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* xs = reinterpret_cast<T*>(smem_raw);                  // [NC][kPatchSlots]
  U* ys = reinterpret_cast<U*>(xs + NC * kPatchSlots);     // [NC][kPatchSlots]
  T* fs = reinterpret_cast<T*>(ys + NC * kPatchSlots);     // [NF][kPatchSlots]
  const int pidx = blockIdx.x;
  const int s0 = m.patch_slot[pidx], ns = m.patch_slot[pidx + 1] - s0, nreg = m.patch_nreg[pidx];
  const int64_t N = m.n_nodes;
  const C* fptr[5] = {cf.phi, cf.u[0], cf.u[1], cf.u[2], cf.mu};
  // CG direction update fused into the gather (CGP): p_new = z + beta p_old with
  // beta = rz_cur / rz_prev; x holds p_old and p_new goes to pout (separate buffers, so that a
  // patch never reads a p value another patch has already updated)
  __shared__ T s_beta;
  if (CGP && threadIdx.x == 0) {
    double bn, bd;
    if (fcg) {
      bn = -S_cg[kFcgAlpha] * S_cg[kFcgZq0 + (par ^ 1)];
      bd = S_cg[kFcgRz0 + (par ^ 1)];
    } else {
      bn = S_cg[kCgRz0 + par];
      bd = S_cg[kCgRzPrev];
    }
    s_beta = (T)(bd != 0.0 ? bn / bd : 0.0);
    if (blockIdx.x == 0) {  // accumulators of the update kernel that follows
      S_cg[kCgRz0 + (par ^ 1)] = 0.0;
      S_cg[kCgRr0 + (par ^ 1)] = 0.0;
    }
  }
  // the element's local corner slots (with its level) are loaded first, so that their latency
  // overlaps the gather of the patch's nodes
  const int64_t e = (int64_t)m.patch_elem[pidx] + threadIdx.x;
  const bool has_elem = e < m.patch_elem[pidx + 1];
  uint4 lp = make_uint4(0, 0, 0, 0);
  if (has_elem) lp = __ldg(m.eloc + e);
  if (CGP) __syncthreads();
  // 1. regular slots
  {
    for (int i = threadIdx.x; i < nreg; i += kPatchElems) {
      const int32_t v = m.slot_node[s0 + i];
      const int64_t g = v & kNodeMask;
      const bool dir = K::DIR && (v & kDirBit);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T xv;
        if (CGP) {
          const S pv = zcg[c * N + g] + (S)s_beta * x[c * N + g];
          pout[c * N + g] = pv;  // patches sharing the node store the same value
          xv = (T)pv;
        } else {
          xv = (T)x[c * N + g];
        }
        xs[c * kPatchSlots + i] = dir ? T(0) : xv;
        ys[c * kPatchSlots + i] = U(0);
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        T val = ldv<T>(fptr[f], g);
        if (f == 0) val += T(cf.phi_shift);
        fs[f * kPatchSlots + i] = val;
      }
    }
  }
  __syncthreads();
  // 2. hanging slots
  for (int i = nreg + threadIdx.x; i < ns; i += blockDim.x) {
    const ushort4 q = m.slot_par[s0 + i];
    const bool four = q.z != 0xffff;
    const T w = four ? T(0.25) : T(0.5);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const T* a = xs + c * kPatchSlots;
      T v = a[q.x] + a[q.y];
      if (four) v += a[q.z] + a[q.w];
      xs[c * kPatchSlots + i] = w * v;
      ys[c * kPatchSlots + i] = U(0);
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      const T* a = fs + f * kPatchSlots;
      T v = a[q.x] + a[q.y];
      if (four) v += a[q.z] + a[q.w];
      fs[f * kPatchSlots + i] = w * v;
    }
  }
  __syncthreads();
  // 3. elements
  typename Acc<T>::type en[1] = {Acc<T>::zero()};
  if (has_elem) {
    const int lev = (int)(lp.x >> kElocLevelShift) & kElocLevelMask;
    const int sl[8] = {(int)(lp.x & kElocSlotMask), (int)(lp.x >> 16), (int)(lp.y & 0xffff),
                       (int)(lp.y >> 16),    (int)(lp.z & 0xffff), (int)(lp.z >> 16),
                       (int)(lp.w & 0xffff), (int)(lp.w >> 16)};
    const Geo<T> g = level_geometry<T>(m, lev);
    T fe[K::NF][8];  // fields the operator ignores are not gathered (zero here)
#pragma unroll
    for (int f = 0; f < K::NF; ++f)
#pragma unroll
      for (int a = 0; a < 8; ++a) fe[f][a] = f < NF ? fs[f * kPatchSlots + sl[a]] : T(0);
    K k;
    k.setup(fe, g, p);
    if constexpr (K::QDATA) k.bind(cf.qd, m.n_elem, e);
    T xin[NC][8];
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int a = 0; a < 8; ++a) xin[c][a] = xs[c * kPatchSlots + sl[a]];
    T r[NC][8];
    constexpr bool EF = PQ && HasEnergy<K>::value;
    if constexpr (EF)
      Acc<T>::add(en[0], k.apply_energy(g, p, xin, r));
    else
      k.apply(g, p, xin, r);
#pragma unroll
    for (int c = 0; c < NC; ++c)
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        if (PQ && !EF) Acc<T>::fma(en[0], xin[c][a], r[c][a]);
        atomicAdd(ys + c * kPatchSlots + sl[a], (U)r[c][a]);
      }
  }
  // p.Ap
  if (PQ) {
    double tot[1];
    block_sum<1, kPatchElems>(en, tot);
    if (threadIdx.x == 0) atomicAdd(S_cg + kCgPq0 + par, tot[0]);
  }
  __syncthreads();
  // 4. hanging slots -> parents
  for (int i = nreg + threadIdx.x; i < ns; i += blockDim.x) {
    const ushort4 q = m.slot_par[s0 + i];
    const bool four = q.z != 0xffff;
    const U w = four ? U(0.25) : U(0.5);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      U* a = ys + c * kPatchSlots;
      const U v = w * a[i];
      atomicAdd(a + q.x, v);
      atomicAdd(a + q.y, v);
      if (four) {
        atomicAdd(a + q.z, v);
        atomicAdd(a + q.w, v);
      }
    }
  }
  __syncthreads();
  // 5. regular slots -> global
  for (int i = threadIdx.x; i < nreg; i += blockDim.x) {
    const int32_t v = m.slot_node[s0 + i];
    if (K::DIR && (v & kDirBit)) continue;
    const int64_t g = v & kNodeMask;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      const S val = (S)ys[c * kPatchSlots + i];
      if (v & kOwnBit)
        y[c * N + g] = val;
      else
        atomic_add(y + c * N + g, val);
    }
  }
}

template <class K, class T>
constexpr size_t patch_smem() {
  return (size_t)(2 * K::NC + gathered_fields<K>()) * kPatchSlots * sizeof(T);
}

// Launch the patch apply, raising the dynamic shared-memory limit once per instantiation.
template <class K, class T, class S, class C, bool PQ, bool CGP = false>
static void launch_patch(const chns_mesh* m, const DevParams& p, const CoefArgs<C>& cf,
                         const S* x, S* y, double* S_cg, cudaStream_t s, const S* z = nullptr,
                         S* pout = nullptr, int par = 0, int fcg = 0) {
  constexpr size_t smem = patch_smem<K, T>();
  static bool configured = false;  // per instantiation
  if (!configured) {
    cudaFuncSetAttribute(k_apply_patch<K, T, S, C, PQ, CGP>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    configured = true;
  }
  note_launch();
  k_apply_patch<K, T, S, C, PQ, CGP><<<(unsigned)m->d.n_patch, kPatchElems, smem, s>>>(
      m->d, p, cf, x, y, S_cg, par, fcg, z, pout);
}

// ---- persistent, software-pipelined patch apply (FP32/FP64 vectors and coefficients of one type).
// Each CTA walks the patches blockIdx.x, blockIdx.x + gridDim.x, ... With the patches of one CTA
// numbered k = 0, 1, ..., iteration k computes patch k (phases 1-5 of k_apply_patch) while
//   - the node values of patch k+1 (x, z for CGP, coefficient fields), its element slot table
//     (with the levels) and the parents of its first kPqStage hanging slots are in flight into
//     the other of two shared-memory stages,
//   - the slot table of patch k+2 is in flight into the third of three index buffers, and
//   - the patch-table entries of patch k+3 are in flight into a ring of four,
// all as cp.async copies, so that no global load of any kind remains in the per-patch chain. The
// sums of PQ are accumulated over all patches of the CTA and added once.
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
template <int B>
__device__ __forceinline__ void cp_async_b(void* dst, const void* src) {
  static_assert(B == 4 || B == 8 || B == 16, "cp.async of 4, 8 or 16 bytes");
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(src), "n"(B) : "memory");
}

constexpr int kPqStage = 128;  // hanging slots per patch whose parents are staged (rest: global)

template <class K, class T, bool CGP>
constexpr int stream_stage_arrays() {
  return (CGP ? 2 : 1) * K::NC + gathered_fields<K>();
}
template <class K, class T, bool CGP>
constexpr size_t stream_smem() {
  // two value stages, the accumulators, three slot-index buffers, two stages of element slot
  // tables and hanging parents, the patch-table ring
  return (size_t)(2 * stream_stage_arrays<K, T, CGP>() + K::NC) * kPatchSlots * sizeof(T) +
         (size_t)3 * kPatchSlots * sizeof(int32_t) + (size_t)2 * kPatchElems * sizeof(uint4) +
         (size_t)2 * kPqStage * sizeof(ushort4) + (size_t)4 * 8 * sizeof(int32_t);
}

template <class K, class T, bool PQ, bool CGP>
__global__ void __launch_bounds__(kPatchElems, K::STREAM_CTAS)
k_apply_stream(MeshDev m, DevParams p, CoefArgs<T> cf, const T* __restrict__ x, T* __restrict__ y,
               double* __restrict__ S_cg, int par, int fcg, const T* __restrict__ zcg,
               T* __restrict__ pout) {
  constexpr int NC = K::NC, NF = gathered_fields<K>(), NA = stream_stage_arrays<K, T, CGP>();
  static_assert(!K::QDATA, "per-element quadrature data is not staged by this kernel");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* vb = reinterpret_cast<T*>(smem_raw);                             // [2][NA][kPatchSlots]
  T* ys = vb + 2 * NA * kPatchSlots;                                  // [NC][kPatchSlots]
  int32_t* ib = reinterpret_cast<int32_t*>(ys + NC * kPatchSlots);    // [3][kPatchSlots]
  uint4* elb = reinterpret_cast<uint4*>(ib + 3 * kPatchSlots);        // [2][kPatchElems]
  ushort4* pqb = reinterpret_cast<ushort4*>(elb + 2 * kPatchElems);   // [2][kPqStage]
  int32_t* mt = reinterpret_cast<int32_t*>(pqb + 2 * kPqStage);
  // mt: [4][8] = first slot, end slot, regular slots, first element, end element
  const int np = (int)m.n_patch, G = gridDim.x, tid = threadIdx.x;
  const int64_t N = m.n_nodes;
  // the arrays gathered per slot, in stage order: x components, z components (CGP), fields
  const T* src_arr[NA];
  {
    const T* fptr[5] = {cf.phi, cf.u[0], cf.u[1], cf.u[2], cf.mu};
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      src_arr[c] = x + c * N;
      if (CGP) src_arr[NC + c] = zcg + c * N;
    }
#pragma unroll
    for (int f = 0; f < NF; ++f) src_arr[(CGP ? 2 : 1) * NC + f] = fptr[f];
  }
  __shared__ T s_beta;
  if (CGP && tid == 0) {
    double bn, bd;
    if (fcg) {
      bn = -S_cg[kFcgAlpha] * S_cg[kFcgZq0 + (par ^ 1)];
      bd = S_cg[kFcgRz0 + (par ^ 1)];
    } else {
      bn = S_cg[kCgRz0 + par];
      bd = S_cg[kCgRzPrev];
    }
    s_beta = (T)(bd != 0.0 ? bn / bd : 0.0);
    if (blockIdx.x == 0) {
      S_cg[kCgRz0 + (par ^ 1)] = 0.0;
      S_cg[kCgRr0 + (par ^ 1)] = 0.0;
    }
  }
  // patch-table entries of patch q into ring entry r (threads 0-4, one word each)
  auto issue_meta = [&](int q, int r) {
    if (tid < 5) {
      const int32_t* src = tid < 2 ? m.patch_slot + q + tid
                                   : tid == 2 ? m.patch_nreg + q : m.patch_elem + q + (tid - 3);
      cp_async_b<4>(mt + 8 * r + tid, src);
    }
  };
  // slot table of patch q (ring entry r landed) into index buffer bi
  auto issue_idx = [&](int r, int bi) {
    const int s0 = mt[8 * r], nr = mt[8 * r + 2];
    int32_t* dst = ib + bi * kPatchSlots;
    for (int i = tid; i < nr; i += kPatchElems) cp_async_b<4>(dst + i, m.slot_node + s0 + i);
  };
  // everything patch q (ring entry r) needs besides its slot table, into stage st: node values
  // (from index buffer bi: each thread reads only entries its own copies wrote), element slot
  // tables, parents of the first kPqStage hanging slots
  auto issue_stage = [&](int r, int st, int bi) {
    const int s0 = mt[8 * r], s1 = mt[8 * r + 1], nr = mt[8 * r + 2];
    const int e0 = mt[8 * r + 3], e1 = mt[8 * r + 4];
    const int32_t* src = ib + bi * kPatchSlots;
    T* dst = vb + st * NA * kPatchSlots;
    for (int i = tid; i < nr; i += kPatchElems) {
      const int g = src[i] & kNodeMask;
#pragma unroll
      for (int a = 0; a < NA; ++a) cp_async_b<sizeof(T)>(dst + a * kPatchSlots + i, src_arr[a] + g);
    }
    if (e0 + tid < e1) cp_async_b<16>(elb + st * kPatchElems + tid, m.eloc + e0 + tid);
    if (tid < kPqStage && nr + tid < s1 - s0)
      cp_async_b<8>(pqb + st * kPqStage + tid, m.slot_par + s0 + nr + tid);
  };
  // prologue: ring entries of patches 0-2, slot tables of patches 0-1, stage 0 of patch 0
  int pid = blockIdx.x;
  for (int j = 0; j < 3; ++j)
    if (pid + j * G < np) issue_meta(pid + j * G, j);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  for (int j = 0; j < 2; ++j)
    if (pid + j * G < np) issue_idx(j, j);
  cp_async_commit();
  cp_async_wait_all();
  __syncthreads();
  if (pid < np) issue_stage(0, 0, 0);
  cp_async_commit();
  // Without Dirichlet rows or the fused CG update the regular slots need no pass of their own:
  // the accumulators are cleared once here and then by the passes that read them (4 and 5), so
  // that every slot is zero again when the next patch starts.
  constexpr bool ZERO_IN_PLACE = !K::DIR && !CGP;
  if constexpr (ZERO_IN_PLACE)
    for (int i = tid; i < NC * kPatchSlots; i += kPatchElems) ys[i] = T(0);
  typename Acc<T>::type en[1] = {Acc<T>::zero()};
  for (int k = 0; pid < np; pid += G, ++k) {
    const int st = k & 1, bc = k % 3, rc = k & 3;
    cp_async_wait_all();
    __syncthreads();  // stage k, slot table k+1 and ring entry k+2 have landed for every thread
    if (pid + G < np) issue_stage((k + 1) & 3, st ^ 1, (k + 1) % 3);
    if (pid + 2 * G < np) issue_idx((k + 2) & 3, (k + 2) % 3);
    if (pid + 3 * G < np) issue_meta(pid + 3 * G, (k + 3) & 3);
    cp_async_commit();
    const int s0 = mt[8 * rc], ns = mt[8 * rc + 1] - s0, nreg = mt[8 * rc + 2];
    const int e0 = mt[8 * rc + 3], ne = mt[8 * rc + 4] - e0;
    T* xs = vb + st * NA * kPatchSlots;
    const T* zs = xs + NC * kPatchSlots;
    T* fs = xs + (CGP ? 2 : 1) * NC * kPatchSlots;
    const int32_t* ic = ib + bc * kPatchSlots;
    const ushort4* pq = pqb + st * kPqStage;
    auto parents = [&](int i) { return i - nreg < kPqStage ? pq[i - nreg] : m.slot_par[s0 + i]; };
    // 1. regular slots: CG direction update, Dirichlet zeros, accumulators cleared
    if constexpr (!ZERO_IN_PLACE) {
      for (int i = tid; i < nreg; i += kPatchElems) {
        const int32_t v = ic[i];
        const bool dir = K::DIR && (v & kDirBit);
#pragma unroll
        for (int c = 0; c < NC; ++c) {
          T xv = xs[c * kPatchSlots + i];
          if (CGP) {
            xv = zs[c * kPatchSlots + i] + s_beta * xv;
            (pout + c * N)[v & kNodeMask] = xv;  // patches sharing the node store the same value
          }
          xs[c * kPatchSlots + i] = dir ? T(0) : xv;
          ys[c * kPatchSlots + i] = T(0);
        }
      }
      __syncthreads();
    }
    // 2. hanging slots
    for (int i = nreg + tid; i < ns; i += kPatchElems) {
      const ushort4 q = parents(i);
      const bool four = q.z != 0xffff;
      const T w = four ? T(0.25) : T(0.5);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T* a = xs + c * kPatchSlots;
        T v = a[q.x] + a[q.y];
        if (four) v += a[q.z] + a[q.w];
        xs[c * kPatchSlots + i] = w * v;
        if (!ZERO_IN_PLACE) ys[c * kPatchSlots + i] = T(0);
      }
#pragma unroll
      for (int f = 0; f < NF; ++f) {
        const T* a = fs + f * kPatchSlots;
        T v = a[q.x] + a[q.y];
        if (four) v += a[q.z] + a[q.w];
        fs[f * kPatchSlots + i] = w * v;
      }
    }
    __syncthreads();
    // 3. elements
    if (tid < ne) {
      const uint4 lp = elb[st * kPatchElems + tid];
      const int lev = (int)(lp.x >> kElocLevelShift) & kElocLevelMask;
      const int sl[8] = {(int)(lp.x & kElocSlotMask), (int)(lp.x >> 16), (int)(lp.y & 0xffff),
                         (int)(lp.y >> 16),    (int)(lp.z & 0xffff), (int)(lp.z >> 16),
                         (int)(lp.w & 0xffff), (int)(lp.w >> 16)};
      const Geo<T> g = level_geometry<T>(m, lev);
      T fe[K::NF][8];  // fields the operator ignores are not gathered (zero here)
#pragma unroll
      for (int f = 0; f < K::NF; ++f)
#pragma unroll
        for (int a = 0; a < 8; ++a) fe[f][a] = f < NF ? fs[f * kPatchSlots + sl[a]] : T(0);
      K kk;
      kk.setup(fe, g, p);
      T xin[NC][8];
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int a = 0; a < 8; ++a) xin[c][a] = xs[c * kPatchSlots + sl[a]];
      T r[NC][8];
      constexpr bool EF = PQ && HasEnergy<K>::value;
      if constexpr (EF)
        Acc<T>::add(en[0], kk.apply_energy(g, p, xin, r));
      else
        kk.apply(g, p, xin, r);
#pragma unroll
      for (int c = 0; c < NC; ++c)
#pragma unroll
        for (int a = 0; a < 8; ++a) {
          if (PQ && !EF) Acc<T>::fma(en[0], xin[c][a], r[c][a]);
          atomicAdd(ys + c * kPatchSlots + sl[a], r[c][a]);
        }
    }
    __syncthreads();
    // 4. hanging slots -> parents
    for (int i = nreg + tid; i < ns; i += kPatchElems) {
      const ushort4 q = parents(i);
      const bool four = q.z != 0xffff;
      const T w = four ? T(0.25) : T(0.5);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        T* a = ys + c * kPatchSlots;
        const T v = w * a[i];
        if (ZERO_IN_PLACE) a[i] = T(0);
        atomicAdd(a + q.x, v);
        atomicAdd(a + q.y, v);
        if (four) {
          atomicAdd(a + q.z, v);
          atomicAdd(a + q.w, v);
        }
      }
    }
    __syncthreads();
    // 5. regular slots -> global (owned: store; shared with other patches: atomic add)
    for (int i = tid; i < nreg; i += kPatchElems) {
      const int32_t v = ic[i];
      if (K::DIR && (v & kDirBit)) continue;
      const int g = v & kNodeMask;
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T val = ys[c * kPatchSlots + i];
        if (ZERO_IN_PLACE) ys[c * kPatchSlots + i] = T(0);
        T* yc = y + c * N;
        if (v & kOwnBit)
          yc[g] = val;
        else
          atomic_add(yc + g, val);
      }
    }
    // the next iteration's first barrier orders these reads before the buffers are refilled
  }
  cp_async_wait_all();
  if (PQ) {
    double tot[1];
    block_sum<1, kPatchElems>(en, tot);
    if (tid == 0) atomicAdd(S_cg + kCgPq0 + par, tot[0]);
  }
}

// Resident CTAs of one instantiation on this device (queried once per instantiation).
template <class Fn>
static int resident_ctas(Fn fn, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kPatchElems, smem) != cudaSuccess)
    per_sm = 1;
  return std::max(per_sm, 1);
}

template <class K, class T, bool PQ, bool CGP>
static void launch_stream(const chns_mesh* m, const DevParams& p, const CoefArgs<T>& cf,
                          const T* x, T* y, double* S_cg, cudaStream_t s, const T* z = nullptr,
                          T* pout = nullptr, int par = 0, int fcg = 0) {
  constexpr size_t smem = stream_smem<K, T, CGP>();
  static int per_sm = 0;  // per instantiation
  if (per_sm == 0) {
    cudaFuncSetAttribute(k_apply_stream<K, T, PQ, CGP>,
                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    per_sm = resident_ctas(k_apply_stream<K, T, PQ, CGP>, smem);
  }
  int64_t grid = (int64_t)per_sm * std::max(m->sm_count, 1);
  if (m->apply_max_ctas > 0) grid = std::min(grid, m->apply_max_ctas);
  grid = std::max<int64_t>(1, std::min(grid, m->d.n_patch));
  note_launch();
  k_apply_stream<K, T, PQ, CGP><<<(unsigned)grid, kPatchElems, smem, s>>>(m->d, p, cf, x, y, S_cg,
                                                                           par, fcg, z, pout);
}

// The persistent kernel pays off once every resident CTA has several patches to walk; operators
// with per-element quadrature data, BF16 coefficients (2-byte copies) and FP64 (ALU bound) keep
// one CTA per patch.
template <class K, class T, class S, class C>
static bool use_stream(const chns_mesh* m) {
  if (!(std::is_same<T, float>::value && std::is_same<S, T>::value && std::is_same<C, T>::value))
    return false;
  if (K::QDATA || K::STREAM_CTAS == 0) return false;
  if (m->apply_kernel == CHNS_APPLY_PATCH) return false;
  if (m->apply_kernel == CHNS_APPLY_STREAM) return true;
  return m->d.n_patch >= (int64_t)kStreamMinPatchesPerSm * std::max(m->sm_count, 1);
}

// Reference (corner a, slot k) -> node reference with Dirichlet bit and its weight, or -1.
__device__ __forceinline__ int corner_ref(const MeshDev& m, int v, int k, double& w) {
  int j = v & kIdxMask;
  if (j < m.n_nodes) {
    w = 1.0;
    return k == 0 ? v : -1;
  }
  int4 h = m.hang[j - m.n_nodes];
  bool four = h.z >= 0;
  w = four ? 0.25 : 0.5;
  int r = k == 0 ? h.x : k == 1 ? h.y : k == 2 ? h.z : h.w;
  return (k >= 2 && !four) ? -1 : r;
}

// Exact diagonal of P^T (sum_e A_e) P: for every node j touching the element (as a corner or as a
// hanging-node parent), apply A_e to the local vector of j's basis function and take its j part.
// BLOCK: the NC x NC nodal block instead, stored as d[(row*NC + col)*N + j].
template <class K, class T, class S, class C, bool BLOCK = false>
__global__ void __launch_bounds__(kApplyThreads) k_diag(MeshDev m, DevParams p, CoefArgs<C> cf,
                                                        S* __restrict__ d) {
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (e >= m.n_elem) return;
  int idx[8];
  load_corners(m, e, idx);
  const Geo<T> g = geometry<T>(m, e);
  K k;
  k.load(m, p, cf, idx, g);
  if constexpr (K::QDATA) k.bind(cf.qd, m.n_elem, e);
  // node references of the 8 corners (a regular corner itself, a hanging corner its 2 or 4
  // parents) and their weights, read once
  int rf[8][4];
  double wt[8][4];
  for (int a = 0; a < 8; ++a)
    for (int s = 0; s < 4; ++s) rf[a][s] = corner_ref(m, idx[a], s, wt[a][s]);
  for (int a = 0; a < 8; ++a) {
    for (int s = 0; s < 4; ++s) {
      const int ref = rf[a][s];
      if (ref < 0) continue;
      if (K::DIR && (ref & kDirBit)) continue;
      const int j = ref & kIdxMask;
      // first occurrence only
      bool seen = false;
      for (int a2 = 0; a2 <= a && !seen; ++a2)
        for (int s2 = 0; s2 < 4; ++s2) {
          if (a2 == a && s2 >= s) break;
          const int r2 = rf[a2][s2];
          if (r2 >= 0 && (r2 & kIdxMask) == j) {
            seen = true;
            break;
          }
        }
      if (seen) continue;
      T lv[8];
      for (int b = 0; b < 8; ++b) {
        T acc = T(0);
        for (int s2 = 0; s2 < 4; ++s2) {
          const int r2 = rf[b][s2];
          if (r2 >= 0 && (r2 & kIdxMask) == j) acc += T(wt[b][s2]);
        }
        lv[b] = acc;
      }
      const int ncd = K::DIAG_PER_COMP ? K::NC : 1;
      for (int c = 0; c < ncd; ++c) {
        T xin[K::NC][8], r[K::NC][8];
        for (int c2 = 0; c2 < K::NC; ++c2)
          for (int b = 0; b < 8; ++b) xin[c2][b] = c2 == c ? lv[b] : T(0);
        k.apply(g, p, xin, r);
        if (BLOCK) {
          for (int r2 = 0; r2 < K::NC; ++r2) {
            T bv = T(0);
            for (int b = 0; b < 8; ++b) bv += lv[b] * r[r2][b];
            atomic_add(d + (r2 * K::NC + c) * m.n_nodes + j, (S)bv);
          }
          continue;
        }
        T dv = T(0);
        for (int b = 0; b < 8; ++b) dv += lv[b] * r[c][b];
        if (K::DIAG_PER_COMP) {
          atomic_add(d + c * m.n_nodes + j, (S)dv);
        } else {
          for (int c2 = 0; c2 < K::NC; ++c2) atomic_add(d + c2 * m.n_nodes + j, (S)dv);
        }
      }
    }
  }
}

// Dirichlet rows: y[c*N + j] = x[c*N + j] (identity) for boundary nodes j.
template <class S>
__global__ void k_dirichlet_copy(const int32_t* __restrict__ bnd, int64_t nb, int64_t N, int nc,
                                 const S* __restrict__ x, S* __restrict__ y) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nb * nc) return;
  const int64_t c = i / nb, j = bnd[i % nb];
  y[c * N + j] = x ? x[c * N + j] : S(1);
}

int op_ncomp(chns_operator op) {
  switch (op) {
    case CHNS_OP_POISSON: return 1;
    case CHNS_OP_MASS: return 3;
    case CHNS_OP_CH: return 2;
    case CHNS_OP_MOMENTUM: return 3;
  }
  return 0;
}
bool op_dirichlet(chns_operator op) { return op == CHNS_OP_MASS || op == CHNS_OP_MOMENTUM; }

template <class C>
static CoefArgs<C> coef_args(const chns_coef* c) {
  CoefArgs<C> a;
  a.phi = static_cast<const C*>(c->phi_tilde);
  for (int d = 0; d < 3; ++d) a.u[d] = static_cast<const C*>(c->u_adv[d]);
  a.mu = static_cast<const C*>(c->mu_tilde);
  a.phi_shift = std::is_same<C, __nv_bfloat16>::value ? -1.0f : 0.0f;
  return a;
}

static chns_status check_coef(chns_operator op, const chns_coef* c) {
  CHNS_CHECK(c && c->phi_tilde, CHNS_EINVAL, "coefficient phi_tilde is required");
  if (op == CHNS_OP_CH || op == CHNS_OP_MOMENTUM)
    CHNS_CHECK(c->u_adv[0] && c->u_adv[1] && c->u_adv[2], CHNS_EINVAL,
               "coefficient u_adv[3] is required");
  if (op == CHNS_OP_MOMENTUM) CHNS_CHECK(c->mu_tilde, CHNS_EINVAL, "coefficient mu_tilde is required");
  return CHNS_OK;
}

template <class T, class S, class C>
static void launch_apply(const chns_mesh* m, chns_operator op, const DevParams& p,
                         const CoefArgs<C>& cf, const S* x, S* y, cudaStream_t s) {
  switch (op) {
    case CHNS_OP_POISSON:
      if constexpr (std::is_same<T, float>::value && std::is_same<S, T>::value &&
                    std::is_same<C, T>::value) {
        if (use_stream<PoissonK<T, C>, T, S, C>(m)) {
          launch_stream<PoissonK<T, C>, T, false, false>(m, p, cf, x, y, nullptr, s);
          break;
        }
      }
      launch_patch<PoissonK<T, C>, T, S, C, false>(m, p, cf, x, y, nullptr, s);
      break;
    case CHNS_OP_MASS:
      if constexpr (std::is_same<T, float>::value && std::is_same<S, T>::value &&
                    std::is_same<C, T>::value) {
        if (use_stream<MassK<T, C>, T, S, C>(m)) {
          launch_stream<MassK<T, C>, T, false, false>(m, p, cf, x, y, nullptr, s);
          break;
        }
      }
      launch_patch<MassK<T, C>, T, S, C, false>(m, p, cf, x, y, nullptr, s);
      break;
    case CHNS_OP_CH:
      launch_patch<ChK<T, C>, T, S, C, false>(m, p, cf, x, y, nullptr, s);
      break;
    case CHNS_OP_MOMENTUM: {
      // quadrature data of the running momentum solve, when it matches this precision
      const void* qd = sizeof(T) == sizeof(double) ? m->mq.qd64 : m->mq.qd32;
      if (m->mq.on && qd) {
        CoefArgs<C> cq = cf;
        cq.qd = qd;
        launch_patch<MomQK<T, C>, T, S, C, false>(m, p, cq, x, y, nullptr, s);
      } else {
        launch_patch<MomK<T, C>, T, S, C, false>(m, p, cf, x, y, nullptr, s);
      }
      break;
    }
  }
}

// The Poisson and mass applies in double-float arithmetic on FP64 arrays.
static void launch_apply_df(const chns_mesh* m, chns_operator op, const DevParams& p,
                            const CoefArgs<double>& cf, const double* x, double* y, cudaStream_t s) {
  if (op == CHNS_OP_POISSON)
    launch_patch<PoissonK<DF, double>, DF, double, double, false>(m, p, cf, x, y, nullptr, s);
  else
    launch_patch<MassK<DF, double>, DF, double, double, false>(m, p, cf, x, y, nullptr, s);
}

// Quadrature data of the momentum operator for the coefficients coef (FP64 and, when coef32 is
// given, FP32), used by every momentum apply until momentum_qdata_off.
chns_status momentum_qdata_on(const chns_mesh* m, const chns_params* prm, const chns_coef* coef64,
                              const chns_coef* coef32, cudaStream_t s) {
  chns_status st = check_coef(CHNS_OP_MOMENTUM, coef64);
  if (st != CHNS_OK) return st;
  const int64_t E = m->d.n_elem;
  const size_t nv = (size_t)8 * kMomQ * E;
  if (!m->mq.qd64) CHNS_CUDA(cudaMalloc(&m->mq.qd64, nv * sizeof(double)));
  if (coef32 && !m->mq.qd32) CHNS_CUDA(cudaMalloc(&m->mq.qd32, nv * sizeof(float)));
  const DevParams p = make_dev_params(*prm);
  const unsigned nb = (unsigned)((E + 127) / 128);
  note_launch();
  k_mom_qdata<double, double><<<nb, 128, 0, s>>>(m->d, p, coef_args<double>(coef64),
                                                 static_cast<double*>(m->mq.qd64));
  if (coef32) {
    note_launch();
    k_mom_qdata<float, float><<<nb, 128, 0, s>>>(m->d, p, coef_args<float>(coef32),
                                                 static_cast<float*>(m->mq.qd32));
  }
  CHNS_CUDA(cudaGetLastError());
  m->mq.on = true;
  m->mq.has32 = coef32 != nullptr;
  return CHNS_OK;
}

void momentum_qdata_off(const chns_mesh* m) { m->mq.on = false; }

template <class T, class S, class C>
static void launch_diag(const chns_mesh* m, chns_operator op, const DevParams& p,
                        const CoefArgs<C>& cf, S* d, cudaStream_t s) {
  const int64_t E = m->d.n_elem;
  const unsigned nb = (unsigned)((E + kApplyThreads - 1) / kApplyThreads);
  switch (op) {
    case CHNS_OP_POISSON:
      note_launch();
      k_diag<PoissonK<T, C>, T, S, C><<<nb, kApplyThreads, 0, s>>>(m->d, p, cf, d);
      break;
    case CHNS_OP_MASS:
      note_launch();
      k_diag<MassK<T, C>, T, S, C><<<nb, kApplyThreads, 0, s>>>(m->d, p, cf, d);
      break;
    case CHNS_OP_CH:
      note_launch();
      k_diag<ChK<T, C>, T, S, C><<<nb, kApplyThreads, 0, s>>>(m->d, p, cf, d);
      break;
    case CHNS_OP_MOMENTUM: {
      note_launch();
      // from the quadrature data of the running momentum solve when it matches this precision
      // (the operator the solve applies; the direct form re-evaluates tau_m per point)
      const void* qd = sizeof(T) == sizeof(double) ? m->mq.qd64 : m->mq.qd32;
      if (m->mq.on && qd) {
        CoefArgs<C> cq = cf;
        cq.qd = qd;
        k_diag<MomQK<T, C>, T, S, C><<<nb, kApplyThreads, 0, s>>>(m->d, p, cq, d);
      } else {
        k_diag<MomK<T, C>, T, S, C><<<nb, kApplyThreads, 0, s>>>(m->d, p, cf, d);
      }
      break;
    }
  }
}

template <class S>
static chns_status dirichlet_rows(const chns_mesh* m, int nc, const S* x, S* y, cudaStream_t s) {
  if (m->n_boundary == 0) return CHNS_OK;
  const int64_t n = m->n_boundary * nc;
  note_launch();
  k_dirichlet_copy<S><<<(unsigned)((n + 255) / 256), 256, 0, s>>>(m->d_bnd, m->n_boundary,
                                                                  m->d.n_nodes, nc, x, y);
  return CHNS_OK;
}

chns_status apply_op(const chns_mesh* m, chns_operator op, const chns_params* prm,
                     const chns_coef* coef, const void* x, void* y, chns_precision prec,
                     cudaStream_t s) {
  CHNS_CHECK(m && prm && x && y, CHNS_EINVAL, "apply: null argument");
  CHNS_CHECK(op >= CHNS_OP_POISSON && op <= CHNS_OP_MOMENTUM, CHNS_EINVAL, "apply: bad operator");
  CHNS_CHECK(x != y, CHNS_EINVAL, "apply: x and y must not alias");
  chns_status st = check_coef(op, coef);
  if (st != CHNS_OK) return st;
  const DevParams p = make_dev_params(*prm);
  const int nc = op_ncomp(op);
  const int64_t n = nc * m->d.n_nodes;
  switch (prec) {
    case CHNS_FP64: {
      CHNS_CUDA(cudaMemsetAsync(y, 0, n * sizeof(double), s));
      launch_apply<double, double, double>(m, op, p, coef_args<double>(coef),
                                           static_cast<const double*>(x), static_cast<double*>(y), s);
      if (op_dirichlet(op))
        dirichlet_rows(m, nc, static_cast<const double*>(x), static_cast<double*>(y), s);
      break;
    }
    case CHNS_FP64_DF: {
      // double-float pays for the light operators (measured on 1.4e6 leaves: Poisson 0.76 ->
      // 0.31 ms, mass 1.01 -> 0.60 ms); the CH and momentum applies are faster in FP64 (1.90 vs
      // 1.96 ms, 7.8 vs 10.1 ms: register pressure and spills)
      CHNS_CUDA(cudaMemsetAsync(y, 0, n * sizeof(double), s));
      if (op == CHNS_OP_POISSON || op == CHNS_OP_MASS)
        launch_apply_df(m, op, p, coef_args<double>(coef), static_cast<const double*>(x),
                        static_cast<double*>(y), s);
      else
        launch_apply<double, double, double>(m, op, p, coef_args<double>(coef),
                                             static_cast<const double*>(x),
                                             static_cast<double*>(y), s);
      if (op_dirichlet(op))
        dirichlet_rows(m, nc, static_cast<const double*>(x), static_cast<double*>(y), s);
      break;
    }
    case CHNS_FP32: {
      CHNS_CUDA(cudaMemsetAsync(y, 0, n * sizeof(float), s));
      launch_apply<float, float, float>(m, op, p, coef_args<float>(coef),
                                        static_cast<const float*>(x), static_cast<float*>(y), s);
      if (op_dirichlet(op))
        dirichlet_rows(m, nc, static_cast<const float*>(x), static_cast<float*>(y), s);
      break;
    }
    case CHNS_FP32_BF16COEF: {
      CHNS_CUDA(cudaMemsetAsync(y, 0, n * sizeof(float), s));
      launch_apply<float, float, __nv_bfloat16>(m, op, p, coef_args<__nv_bfloat16>(coef),
                                                static_cast<const float*>(x),
                                                static_cast<float*>(y), s);
      if (op_dirichlet(op))
        dirichlet_rows(m, nc, static_cast<const float*>(x), static_cast<float*>(y), s);
      break;
    }
    default:
      set_error("apply: bad precision");
      return CHNS_EINVAL;
  }
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

// The operator K with its Dirichlet rows and columns kept (the lifting of Dirichlet data).
template <class K>
struct NoDirK : K {
  static constexpr bool DIR = false;
};

chns_status apply_op_full(const chns_mesh* m, chns_operator op, const chns_params* prm,
                          const chns_coef* coef, const double* x, double* y, cudaStream_t s) {
  CHNS_CHECK(m && prm && x && y && x != y && (op == CHNS_OP_MASS || op == CHNS_OP_MOMENTUM),
             CHNS_EINVAL, "apply without Dirichlet rows: bad argument");
  chns_status st = check_coef(op, coef);
  if (st != CHNS_OK) return st;
  const DevParams p = make_dev_params(*prm);
  CHNS_CUDA(cudaMemsetAsync(y, 0, 3 * m->d.n_nodes * sizeof(double), s));
  if (op == CHNS_OP_MASS)
    launch_patch<NoDirK<MassK<double, double>>, double, double, double, false>(
        m, p, coef_args<double>(coef), x, y, nullptr, s);
  else
    launch_patch<NoDirK<MomK<double, double>>, double, double, double, false>(
        m, p, coef_args<double>(coef), x, y, nullptr, s);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

chns_status dirichlet_set(const chns_mesh* m, int nc, const double* x, double* y, cudaStream_t s) {
  CHNS_CHECK(m && x && y, CHNS_EINVAL, "dirichlet_set: null argument");
  dirichlet_rows<double>(m, nc, x, y, s);
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

chns_status diag_op(const chns_mesh* m, chns_operator op, const chns_params* prm,
                    const chns_coef* coef, void* d, chns_precision prec, cudaStream_t s) {
  CHNS_CHECK(m && prm && d, CHNS_EINVAL, "diagonal: null argument");
  CHNS_CHECK(op >= CHNS_OP_POISSON && op <= CHNS_OP_MOMENTUM, CHNS_EINVAL, "diagonal: bad operator");
  chns_status st = check_coef(op, coef);
  if (st != CHNS_OK) return st;
  const DevParams p = make_dev_params(*prm);
  const int nc = op_ncomp(op);
  const int64_t n = nc * m->d.n_nodes;
  switch (prec) {
    case CHNS_FP64:
      CHNS_CUDA(cudaMemsetAsync(d, 0, n * sizeof(double), s));
      launch_diag<double, double, double>(m, op, p, coef_args<double>(coef),
                                          static_cast<double*>(d), s);
      if (op_dirichlet(op)) dirichlet_rows<double>(m, nc, nullptr, static_cast<double*>(d), s);
      break;
    case CHNS_FP32:
      CHNS_CUDA(cudaMemsetAsync(d, 0, n * sizeof(float), s));
      launch_diag<float, float, float>(m, op, p, coef_args<float>(coef), static_cast<float*>(d), s);
      if (op_dirichlet(op)) dirichlet_rows<float>(m, nc, nullptr, static_cast<float*>(d), s);
      break;
    case CHNS_FP32_BF16COEF:
      CHNS_CUDA(cudaMemsetAsync(d, 0, n * sizeof(float), s));
      launch_diag<float, float, __nv_bfloat16>(m, op, p, coef_args<__nv_bfloat16>(coef),
                                               static_cast<float*>(d), s);
      if (op_dirichlet(op)) dirichlet_rows<float>(m, nc, nullptr, static_cast<float*>(d), s);
      break;
    default:
      set_error("diagonal: bad precision");
      return CHNS_EINVAL;
  }
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

chns_status apply_poisson_cg(const chns_mesh* m, const chns_params* prm, const chns_coef* coef,
                             const void* z, const void* p_old, void* p_new, void* y,
                             chns_precision prec, double* S_cg, int par, cudaStream_t s,
                             bool fcg) {
  chns_status st = check_coef(CHNS_OP_POISSON, coef);
  if (st != CHNS_OK) return st;
  const DevParams p = make_dev_params(*prm);
  switch (prec) {
    case CHNS_FP64:
      launch_patch<PoissonK<double, double>, double, double, double, true, true>(
          m, p, coef_args<double>(coef), static_cast<const double*>(p_old),
          static_cast<double*>(y), S_cg, s, static_cast<const double*>(z),
          static_cast<double*>(p_new), par, fcg);
      break;
    case CHNS_FP32:
      if (use_stream<PoissonK<float, float>, float, float, float>(m)) {
        launch_stream<PoissonK<float, float>, float, true, true>(
            m, p, coef_args<float>(coef), static_cast<const float*>(p_old), static_cast<float*>(y),
            S_cg, s, static_cast<const float*>(z), static_cast<float*>(p_new), par, fcg);
        break;
      }
      launch_patch<PoissonK<float, float>, float, float, float, true, true>(
          m, p, coef_args<float>(coef), static_cast<const float*>(p_old), static_cast<float*>(y),
          S_cg, s, static_cast<const float*>(z), static_cast<float*>(p_new), par, fcg);
      break;
    case CHNS_FP32_BF16COEF:
      launch_patch<PoissonK<float, __nv_bfloat16>, float, float, __nv_bfloat16, true, true>(
          m, p, coef_args<__nv_bfloat16>(coef), static_cast<const float*>(p_old),
          static_cast<float*>(y), S_cg, s, static_cast<const float*>(z), static_cast<float*>(p_new),
          par, fcg);
      break;
    default:
      set_error("apply: bad precision");
      return CHNS_EINVAL;
  }
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

// y = sa M x + sb K x and its exact diagonal (shifted Laplacian, constant coefficients); phi is
// any coefficient array of the precision (gathered by the patch kernel, not used).
static DevParams shift_params(const chns_params* prm, double sa, double sb) {
  DevParams p = make_dev_params(*prm);
  p.d.sa = sa;
  p.d.sb = sb;
  p.f.sa = (float)sa;
  p.f.sb = (float)sb;
  return p;
}

chns_status apply_shift(const chns_mesh* m, const chns_params* prm, const void* phi, double sa,
                        double sb, const void* x, void* y, chns_precision prec, cudaStream_t s) {
  CHNS_CHECK(m && prm && phi && x && y && x != y, CHNS_EINVAL, "shifted apply: bad argument");
  const DevParams p = shift_params(prm, sa, sb);
  chns_coef c{};
  c.phi_tilde = phi;
  const int64_t N = m->d.n_nodes;
  if (prec == CHNS_FP64) {
    CHNS_CUDA(cudaMemsetAsync(y, 0, N * sizeof(double), s));
    launch_patch<ShiftK<double, double>, double, double, double, false>(
        m, p, coef_args<double>(&c), static_cast<const double*>(x), static_cast<double*>(y),
        nullptr, s);
  } else if (prec == CHNS_FP32) {
    CHNS_CUDA(cudaMemsetAsync(y, 0, N * sizeof(float), s));
    if (use_stream<ShiftK<float, float>, float, float, float>(m))
      launch_stream<ShiftK<float, float>, float, false, false>(
          m, p, coef_args<float>(&c), static_cast<const float*>(x), static_cast<float*>(y),
          nullptr, s);
    else
      launch_patch<ShiftK<float, float>, float, float, float, false>(
          m, p, coef_args<float>(&c), static_cast<const float*>(x), static_cast<float*>(y),
          nullptr, s);
  } else {
    set_error("shifted apply: bad precision");
    return CHNS_EINVAL;
  }
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

chns_status diag_shift(const chns_mesh* m, const chns_params* prm, const void* phi, double sa,
                       double sb, void* d, chns_precision prec, cudaStream_t s) {
  CHNS_CHECK(m && prm && phi && d, CHNS_EINVAL, "shifted diagonal: bad argument");
  const DevParams p = shift_params(prm, sa, sb);
  chns_coef c{};
  c.phi_tilde = phi;
  const int64_t N = m->d.n_nodes;
  const unsigned nb = (unsigned)((m->d.n_elem + kApplyThreads - 1) / kApplyThreads);
  note_launch();
  if (prec == CHNS_FP64) {
    CHNS_CUDA(cudaMemsetAsync(d, 0, N * sizeof(double), s));
    k_diag<ShiftK<double, double>, double, double, double><<<nb, kApplyThreads, 0, s>>>(
        m->d, p, coef_args<double>(&c), static_cast<double*>(d));
  } else if (prec == CHNS_FP32) {
    CHNS_CUDA(cudaMemsetAsync(d, 0, N * sizeof(float), s));
    k_diag<ShiftK<float, float>, float, float, float><<<nb, kApplyThreads, 0, s>>>(
        m->d, p, coef_args<float>(&c), static_cast<float*>(d));
  } else {
    set_error("shifted diagonal: bad precision");
    return CHNS_EINVAL;
  }
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

// 2x2 nodal blocks of the CH Jacobian, d4 = [d_pp, d_pm, d_mp, d_mm] x N, in FP64 or FP32.
chns_status block_diag_ch(const chns_mesh* m, const chns_params* prm, const chns_coef* coef,
                          void* d4, chns_precision prec, cudaStream_t s) {
  chns_status st = check_coef(CHNS_OP_CH, coef);
  if (st != CHNS_OK) return st;
  const DevParams p = make_dev_params(*prm);
  const unsigned nb = (unsigned)((m->d.n_elem + kApplyThreads - 1) / kApplyThreads);
  note_launch();
  if (prec == CHNS_FP64) {
    CHNS_CUDA(cudaMemsetAsync(d4, 0, 4 * m->d.n_nodes * sizeof(double), s));
    k_diag<ChK<double, double>, double, double, double, true>
        <<<nb, kApplyThreads, 0, s>>>(m->d, p, coef_args<double>(coef), static_cast<double*>(d4));
  } else if (prec == CHNS_FP32) {
    CHNS_CUDA(cudaMemsetAsync(d4, 0, 4 * m->d.n_nodes * sizeof(float), s));
    k_diag<ChK<float, float>, float, float, float, true>
        <<<nb, kApplyThreads, 0, s>>>(m->d, p, coef_args<float>(coef), static_cast<float*>(d4));
  } else {
    set_error("block diagonal: bad precision");
    return CHNS_EINVAL;
  }
  CHNS_CUDA(cudaGetLastError());
  return CHNS_OK;
}

}  // namespace chns

using namespace chns;

extern "C" chns_status chns_apply_poisson(const chns_mesh* m, const chns_params* prm,
                                          const chns_coef* coef, const void* x, void* y,
                                          chns_precision prec, void* stream) {
  return apply_op(m, CHNS_OP_POISSON, prm, coef, x, y, prec, as_stream(stream));
}
extern "C" chns_status chns_apply_mass(const chns_mesh* m, const chns_params* prm,
                                       const chns_coef* coef, const void* x, void* y,
                                       chns_precision prec, void* stream) {
  return apply_op(m, CHNS_OP_MASS, prm, coef, x, y, prec, as_stream(stream));
}
extern "C" chns_status chns_apply_ch(const chns_mesh* m, const chns_params* prm,
                                     const chns_coef* coef, const void* x, void* y,
                                     chns_precision prec, void* stream) {
  return apply_op(m, CHNS_OP_CH, prm, coef, x, y, prec, as_stream(stream));
}
extern "C" chns_status chns_apply_momentum(const chns_mesh* m, const chns_params* prm,
                                           const chns_coef* coef, const void* x, void* y,
                                           chns_precision prec, void* stream) {
  return apply_op(m, CHNS_OP_MOMENTUM, prm, coef, x, y, prec, as_stream(stream));
}
extern "C" chns_status chns_operator_diagonal(const chns_mesh* m, chns_operator op,
                                              const chns_params* prm, const chns_coef* coef,
                                              void* d, chns_precision prec, void* stream) {
  return diag_op(m, op, prm, coef, d, prec, as_stream(stream));
}
