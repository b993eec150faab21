// Mesh construction: validation of the leaf list, node enumeration, hanging-node detection and
// upload of the device tables (Sec. 5.2 "Octree construction and 2:1 balancing" and Sec. 5.3
// "Identification of unique, independent nodes").
//
// Instead of the paper's distributed sort of (element, node) edges, this builds flat index tables
// once on the host: every leaf emits its 8 corners (candidate nodes) and its 12 edge midpoints and
// 6 face centres ("cancellation" positions one level deeper). A corner that coincides with a
// cancellation position of some leaf lies inside that leaf's edge or face and is hanging; its
// parents are that edge's two ends (weight 1/2) or that face's four corners (weight 1/4), the
// interpolation from the immediate parent of Fig. "traversal". Under the full 2:1 balance the
// parents of a hanging node are never hanging themselves; this is checked.
#include <algorithm>
#include <array>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

#include "internal.h"
#include "hostutil.h"

namespace chns {
namespace {

using host::compact3;
using host::kFull;
using host::morton;
using host::parallel_for;

struct Cancel {
  uint64_t key;      // Morton key of the midpoint/centre
  int32_t leaf;
  int32_t kind;      // 0..11 edges, 12..17 faces
  bool operator<(const Cancel& o) const { return key < o.key; }
};

// Corner c (0..7, bits x,y,z) of a leaf.
inline void corner_xyz(const uint32_t* a, uint64_t s, int c, uint64_t out[3]) {
  out[0] = a[0] + ((c & 1) ? s : 0);
  out[1] = a[1] + (((c >> 1) & 1) ? s : 0);
  out[2] = a[2] + (((c >> 2) & 1) ? s : 0);
}

// Cancellation position `kind` of a leaf and its parent corners (2 for edges, 4 for faces).
// Edges: kind = 4*d + (b1 + 2*b2): axis d, offsets b1,b2 on the two other axes (ascending).
// Faces: kind = 12 + 2*d + b: normal axis d at side b.
inline int cancel_geom(int kind, int par[4], int mid_half[3], int base_bits[3]) {
  if (kind < 12) {
    int d = kind / 4, r = kind % 4;
    int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
    int b1 = r & 1, b2 = r >> 1;
    base_bits[0] = base_bits[1] = base_bits[2] = 0;
    base_bits[o1] = b1;
    base_bits[o2] = b2;
    mid_half[0] = mid_half[1] = mid_half[2] = 0;
    mid_half[d] = 1;
    int c0 = base_bits[0] | (base_bits[1] << 1) | (base_bits[2] << 2);
    par[0] = c0;
    par[1] = c0 | (1 << d);
    par[2] = par[3] = -1;
    return 2;
  }
  int f = kind - 12, d = f / 2, b = f % 2;
  int o1 = d == 0 ? 1 : 0, o2 = d == 2 ? 1 : 2;
  base_bits[0] = base_bits[1] = base_bits[2] = 0;
  base_bits[d] = b;
  mid_half[0] = mid_half[1] = mid_half[2] = 1;
  mid_half[d] = 0;
  int c0 = b << d;
  par[0] = c0;
  par[1] = c0 | (1 << o1);
  par[2] = c0 | (1 << o2);
  par[3] = c0 | (1 << o1) | (1 << o2);
  return 4;
}

}  // namespace

static chns_status alloc_workspace(chns_mesh* m, bool light) {
  const int64_t N = m->d.n_nodes;
  const size_t n3 = (size_t)(3 * N);
  Workspace& w = m->ws;
  if (light) {
    // level meshes of a multigrid hierarchy: operator applies and diagonals only (no Krylov
    // solve runs on them), so no solver vectors
    CHNS_CUDA(cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
    return CHNS_OK;
  }
  w.v64.assign(kNumVec64, nullptr);
  w.v32.assign(kNumVec32, nullptr);
  for (auto& p : w.v64) CHNS_CUDA(cudaMalloc(&p, n3 * sizeof(double)));
  for (auto& p : w.v32) CHNS_CUDA(cudaMalloc(&p, n3 * sizeof(float)));
  CHNS_CUDA(cudaMalloc(&w.gm_V, (size_t)(CHNS_GMRES_MAX_RESTART + 1) * n3 * sizeof(double)));
  CHNS_CUDA(cudaMalloc(&w.gm_V32, (size_t)(CHNS_GMRES_MAX_RESTART + 1) * n3 * sizeof(float)));
  CHNS_CUDA(cudaMalloc(&w.red, (size_t)(kScalarBase + 1024) * sizeof(double)));
  CHNS_CUDA(cudaMemset(w.red, 0, (size_t)(kScalarBase + 1024) * sizeof(double)));
  CHNS_CUDA(cudaMalloc(&w.counter, 64 * sizeof(unsigned int)));
  CHNS_CUDA(cudaMemset(w.counter, 0, 64 * sizeof(unsigned int)));
  CHNS_CUDA(cudaMallocHost(&w.h_pinned, 1024 * sizeof(double)));
  CHNS_CUDA(cudaMalloc(&w.coef32, (size_t)10 * N * sizeof(float)));
  CHNS_CUDA(cudaMalloc(&w.coef16, (size_t)8 * N * sizeof(__nv_bfloat16)));
  CHNS_CUDA(cudaMalloc(&w.coef64, (size_t)16 * N * sizeof(double)));
  CHNS_CUDA(cudaMalloc(&w.part_big, (size_t)(m->d.n_elem / 64 + 64) * sizeof(double)));
  CHNS_CUDA(cudaMalloc(&w.md_part,
                       (size_t)(CHNS_GMRES_MAX_RESTART + 2) * kMdMaxBlocks * sizeof(double)));
  CHNS_CUDA(cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking));
  return CHNS_OK;
}

static void dfree(void* p) {
  if (p) cudaFree(p);
}

void free_mesh(chns_mesh* m) {
  if (!m) return;
  dfree(m->d_enode);
  dfree(m->d_level);
  dfree(m->d_hang);
  dfree(m->d_anchor);
  dfree(m->d_bnd);
  dfree(m->d_patch_elem);
  dfree(m->d_patch_slot);
  dfree(m->d_patch_nreg);
  dfree(m->d_slot_node);
  dfree(m->d_slot_par);
  dfree(m->d_eloc);
  dfree(m->d_geo);
  dfree(m->d_node_int);
  Workspace& w = m->ws;
  for (auto p : w.v64) dfree(p);
  for (auto p : w.v32) dfree(p);
  dfree(w.gm_V);
  dfree(w.gm_V32);
  dfree(w.red);
  dfree(w.counter);
  if (w.h_pinned) cudaFreeHost(w.h_pinned);
  dfree(w.coef32);
  dfree(w.coef16);
  dfree(w.coef64);
  dfree(w.part_big);
  dfree(w.md_part);
  dfree(m->mq.qd64);
  dfree(m->mq.qd32);
  for (int p = 0; p < 2; ++p)
    for (int k = 0; k < 2; ++k) dfree(m->sd.d[p][k]);
  dfree(m->qvu);
  if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
  delete m;
}

// Greedy partition of the Morton-ordered elements into patches (see kPatchElems/kPatchSlots):
// regular slots = distinct nodes used as corners or as parents of hanging corners, hanging slots
// = distinct hanging corners; a node is owned by a patch when no other patch has it as a slot.
struct PatchTables {
  std::vector<int32_t> elem, slot, nreg, node;
  std::vector<ushort4> par;
  std::vector<uint4> eloc;
};

static_assert(kPatchSlots - 1 <= (int)kElocSlotMask && CHNS_MAXD - 1 <= (int)kElocLevelMask &&
                  kElocLevelShift + 5 <= 16,
              "patch slot and level must fit the first uint16 of eloc");

static void build_patches(int64_t n, int64_t N, const std::vector<int32_t>& enode,
                          const std::vector<int4>& hang, const uint8_t* levels, PatchTables& P) {
  std::vector<int32_t> stamp_n(N, -1), slot_n(N, 0), stamp_h(hang.size(), -1), slot_h(hang.size(), 0);
  std::vector<int32_t> count(N, 0);
  std::vector<int32_t> reg, hg;                    // current patch: node ids, hanging ids
  std::vector<std::array<int32_t, 8>> ecorner;     // provisional: >= 0 regular slot, < 0 ~hslot
  int32_t pid = 0;
  int64_t e0 = 0;
  P.eloc.resize(n);
  auto close = [&](int64_t e_end) {
    const int32_t nr = (int32_t)reg.size();
    P.elem.push_back((int32_t)e0);
    P.slot.push_back((int32_t)P.node.size());
    P.nreg.push_back(nr);
    for (int32_t id : reg) {
      P.node.push_back(id);
      P.par.push_back(make_ushort4(0xffff, 0xffff, 0xffff, 0xffff));
      ++count[id & kIdxMask & ~kDirBit];
    }
    for (int32_t h : hg) {
      const int4 q = hang[h];
      const int32_t ps[4] = {q.x, q.y, q.z, q.w};
      unsigned short loc[4] = {0xffff, 0xffff, 0xffff, 0xffff};
      for (int k = 0; k < 4; ++k)
        if (ps[k] >= 0) loc[k] = (unsigned short)slot_n[ps[k] & kIdxMask];
      P.node.push_back(-1);
      P.par.push_back(make_ushort4(loc[0], loc[1], loc[2], loc[3]));
    }
    for (int64_t e = e0; e < e_end; ++e) {
      unsigned short l[8];
      for (int c = 0; c < 8; ++c) {
        int32_t v = ecorner[e - e0][c];
        l[c] = (unsigned short)(v >= 0 ? v : nr + ~v);
      }
      l[0] = (unsigned short)(l[0] | ((uint32_t)levels[e] << kElocLevelShift));
      P.eloc[e] = make_uint4(l[0] | (l[1] << 16), l[2] | (l[3] << 16), l[4] | (l[5] << 16),
                             l[6] | (l[7] << 16));
    }
    reg.clear();
    hg.clear();
    ecorner.clear();
    ++pid;
    e0 = e_end;
  };
  for (int64_t e = 0; e < n; ++e) {
    // distinct new references of this element
    int32_t newn[40], newh[8];
    int nn = 0, nh = 0;
    auto add_node = [&](int32_t id) {
      const int32_t j = id & kIdxMask;
      if (stamp_n[j] == pid) return;
      for (int k = 0; k < nn; ++k)
        if ((newn[k] & kIdxMask) == j) return;
      newn[nn++] = id;
    };
    for (int c = 0; c < 8; ++c) {
      const int32_t v = enode[8 * e + c];
      const int32_t j = v & kIdxMask;
      if (j < N) {
        add_node(v);
      } else {
        const int32_t h = j - (int32_t)N;
        bool seen = stamp_h[h] == pid;
        for (int k = 0; k < nh && !seen; ++k) seen = newh[k] == h;
        if (!seen) newh[nh++] = h;
        const int4 q = hang[h];
        add_node(q.x);
        add_node(q.y);
        if (q.z >= 0) {
          add_node(q.z);
          add_node(q.w);
        }
      }
    }
    const int64_t slots = (int64_t)reg.size() + hg.size() + nn + nh;
    if (e > e0 && (e - e0 >= kPatchElems || slots > kPatchSlots)) {
      close(e);
      --e;  // re-examine this element in the new patch
      continue;
    }
    for (int k = 0; k < nn; ++k) {
      const int32_t j = newn[k] & kIdxMask;
      stamp_n[j] = pid;
      slot_n[j] = (int32_t)reg.size();
      reg.push_back(newn[k]);
    }
    for (int k = 0; k < nh; ++k) {
      stamp_h[newh[k]] = pid;
      slot_h[newh[k]] = (int32_t)hg.size();
      hg.push_back(newh[k]);
    }
    std::array<int32_t, 8> ec;
    for (int c = 0; c < 8; ++c) {
      const int32_t j = enode[8 * e + c] & kIdxMask;
      ec[c] = j < N ? slot_n[j] : ~slot_h[j - (int32_t)N];
    }
    ecorner.push_back(ec);
  }
  close(n);
  P.elem.push_back((int32_t)n);
  P.slot.push_back((int32_t)P.node.size());
  for (auto& id : P.node)
    if (id >= 0 && count[id & kIdxMask & ~kDirBit] == 1) id |= kOwnBit;
}

chns_status build_mesh(const uint32_t* anchors, const uint8_t* levels, int64_t n,
                       const double extent[3], cudaStream_t stream, chns_mesh* m, bool light,
                       bool keep_host) {
  CHNS_CHECK(n > 0 && n < (int64_t(1) << 28), CHNS_EINVAL, "n_leaves out of range");
  for (int d = 0; d < 3; ++d)
    CHNS_CHECK(extent[d] > 0.0, CHNS_EINVAL, "extent must be positive");

  // ---- per-leaf checks: level range, alignment, Morton order, disjointness, coverage
  std::vector<uint64_t> lkey(n);
  int minl = CHNS_MAXD, maxl = 0;
  for (int64_t i = 0; i < n; ++i) {
    int l = levels[i];
    CHNS_CHECK(l < CHNS_MAXD, CHNS_EINVAL, "leaf level must be < CHNS_MAXD");
    uint64_t s = kFull >> l;
    for (int d = 0; d < 3; ++d) {
      uint64_t a = anchors[3 * i + d];
      CHNS_CHECK(a % s == 0 && a + s <= kFull, CHNS_EINVAL, "anchor not aligned or outside the cube");
    }
    lkey[i] = morton(anchors[3 * i], anchors[3 * i + 1], anchors[3 * i + 2]);
    minl = std::min(minl, l);
    maxl = std::max(maxl, l);
  }
  unsigned __int128 vol = 0;
  for (int64_t i = 0; i < n; ++i) {
    uint64_t span = 1ull << (3 * (CHNS_MAXD - levels[i]));
    vol += span;
    if (i + 1 < n)
      CHNS_CHECK(lkey[i] + span <= lkey[i + 1], CHNS_EINVAL,
                 "leaves are not in strictly increasing Morton order or overlap");
  }
  CHNS_CHECK(vol == ((unsigned __int128)1 << (3 * CHNS_MAXD)), CHNS_EINVAL,
             "leaves do not cover the unit cube");

  // ---- 2:1 balance across faces, edges and corners: the same-size neighbour in each of the 26
  // directions must lie in a leaf at most one level coarser.
  std::atomic<bool> unbalanced(false);
  parallel_for(n, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e && !unbalanced.load(); ++i) {
      int l = levels[i];
      int64_t s = int64_t(kFull >> l);
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            if (!dx && !dy && !dz) continue;
            int64_t p[3] = {int64_t(anchors[3 * i]) + dx * s + s / 2,
                            int64_t(anchors[3 * i + 1]) + dy * s + s / 2,
                            int64_t(anchors[3 * i + 2]) + dz * s + s / 2};
            if (p[0] < 0 || p[1] < 0 || p[2] < 0 || p[0] >= int64_t(kFull) ||
                p[1] >= int64_t(kFull) || p[2] >= int64_t(kFull))
              continue;
            uint64_t k = morton(p[0], p[1], p[2]);
            int64_t j = int64_t(std::upper_bound(lkey.begin(), lkey.end(), k) - lkey.begin()) - 1;
            if (j < 0 || int(levels[j]) < l - 1) unbalanced.store(true);
          }
    }
  });
  CHNS_CHECK(!unbalanced.load(), CHNS_EUNBALANCED, "leaves are not 2:1 balanced");

  // ---- unique corner points
  std::vector<uint64_t> ckey((size_t)n * 8);
  parallel_for(n, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      uint64_t s = kFull >> levels[i];
      for (int c = 0; c < 8; ++c) {
        uint64_t q[3];
        corner_xyz(anchors + 3 * i, s, c, q);
        ckey[8 * i + c] = morton(q[0], q[1], q[2]);
      }
    }
  });
  std::vector<uint64_t> pts(ckey);
  std::sort(pts.begin(), pts.end());
  pts.erase(std::unique(pts.begin(), pts.end()), pts.end());
  const int64_t NP = (int64_t)pts.size();

  // ---- cancellation positions and hanging detection
  std::vector<Cancel> canc((size_t)n * 18);
  parallel_for(n, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i) {
      uint64_t s = kFull >> levels[i], h = s / 2;
      for (int k = 0; k < 18; ++k) {
        int par[4], mh[3], bb[3];
        cancel_geom(k, par, mh, bb);
        uint64_t q[3];
        for (int d = 0; d < 3; ++d) q[d] = anchors[3 * i + d] + bb[d] * s + mh[d] * h;
        canc[18 * i + k] = Cancel{morton(q[0], q[1], q[2]), (int32_t)i, (int32_t)k};
      }
    }
  });
  std::sort(canc.begin(), canc.end());
  std::vector<int32_t> hang_src(NP, -1);   // index into canc of a cancellation at this point
  parallel_for(NP, [&](int64_t b, int64_t e) {
    for (int64_t p = b; p < e; ++p) {
      auto it = std::lower_bound(canc.begin(), canc.end(), Cancel{pts[p], 0, 0});
      if (it != canc.end() && it->key == pts[p]) hang_src[p] = int32_t(it - canc.begin());
    }
  });

  // ---- numbering: independent nodes in Morton order (pts is sorted by Morton key)
  std::vector<int64_t> pid(NP);
  int64_t N = 0, H = 0;
  for (int64_t p = 0; p < NP; ++p) pid[p] = hang_src[p] < 0 ? N++ : -(++H);
  CHNS_CHECK(N < (int64_t(1) << 29) && H < (int64_t(1) << 29), CHNS_EINVAL, "mesh too large");

  auto point_index = [&](uint64_t key) -> int64_t {
    auto it = std::lower_bound(pts.begin(), pts.end(), key);
    if (it == pts.end() || *it != key) return -1;
    return int64_t(it - pts.begin());
  };

  m->node_coords.resize((size_t)3 * N);
  m->node_bnd.resize((size_t)N);
  int64_t nb = 0;
  for (int64_t p = 0; p < NP; ++p) {
    if (pid[p] < 0) continue;
    uint64_t x = compact3(pts[p]), y = compact3(pts[p] >> 1), z = compact3(pts[p] >> 2);
    int64_t j = pid[p];
    m->node_coords[3 * j] = (uint32_t)x;
    m->node_coords[3 * j + 1] = (uint32_t)y;
    m->node_coords[3 * j + 2] = (uint32_t)z;
    bool b = x == 0 || y == 0 || z == 0 || x == kFull || y == kFull || z == kFull;
    m->node_bnd[j] = b ? 1 : 0;
    nb += b;
  }
  auto flagged = [&](int64_t j) -> int32_t {
    return (int32_t)j | (m->node_bnd[j] ? kDirBit : 0);
  };

  // hanging table
  std::vector<int4> hang((size_t)std::max<int64_t>(H, 1));
  bool bad = false;
  for (int64_t p = 0; p < NP; ++p) {
    if (pid[p] >= 0) continue;
    int64_t h = -pid[p] - 1;
    const Cancel& c = canc[hang_src[p]];
    int par[4], mh[3], bb[3];
    int np = cancel_geom(c.kind, par, mh, bb);
    uint64_t s = kFull >> levels[c.leaf];
    int32_t out[4] = {-1, -1, -1, -1};
    for (int k = 0; k < np; ++k) {
      uint64_t q[3];
      corner_xyz(anchors + 3 * c.leaf, s, par[k], q);
      int64_t pp = point_index(morton(q[0], q[1], q[2]));
      if (pp < 0 || pid[pp] < 0) {
        bad = true;
        break;
      }
      out[k] = flagged(pid[pp]);
    }
    hang[h] = make_int4(out[0], out[1], out[2], out[3]);
  }
  CHNS_CHECK(!bad, CHNS_EUNBALANCED, "hanging node whose parent is not an independent node");

  // element corner table
  std::vector<int32_t> enode((size_t)n * 8);
  parallel_for(n, [&](int64_t b, int64_t e) {
    for (int64_t i = b; i < e; ++i)
      for (int c = 0; c < 8; ++c) {
        int64_t p = point_index(ckey[8 * i + c]);
        int64_t id = pid[p];
        enode[8 * i + c] = id >= 0 ? flagged(id) : (int32_t)(N + (-id - 1));
      }
  });

  if (keep_host) {
    m->h_enode = enode;
    m->h_hang.assign(hang.begin(), hang.begin() + H);
  }

  // ---- patches (CTA-level gather / scatter)
  PatchTables P;
  build_patches(n, N, enode, hang, levels, P);

  // ---- upload
  m->d.n_elem = n;
  m->d.n_nodes = N;
  m->d.n_hang = H;
  for (int d = 0; d < 3; ++d) m->d.ext[d] = extent[d];
  m->min_level = minl;
  m->max_level = maxl;
  m->n_boundary = nb;
  CHNS_CUDA(cudaMalloc(&m->d_enode, (size_t)n * 8 * sizeof(int32_t)));
  CHNS_CUDA(cudaMalloc(&m->d_level, (size_t)n));
  CHNS_CUDA(cudaMalloc(&m->d_hang, hang.size() * sizeof(int4)));
  CHNS_CUDA(cudaMalloc(&m->d_anchor, (size_t)n * 3 * sizeof(uint32_t)));
  CHNS_CUDA(cudaMemcpyAsync(m->d_enode, enode.data(), (size_t)n * 8 * sizeof(int32_t),
                            cudaMemcpyHostToDevice, stream));
  CHNS_CUDA(cudaMemcpyAsync(m->d_level, levels, (size_t)n, cudaMemcpyHostToDevice, stream));
  CHNS_CUDA(cudaMemcpyAsync(m->d_hang, hang.data(), hang.size() * sizeof(int4),
                            cudaMemcpyHostToDevice, stream));
  CHNS_CUDA(cudaMemcpyAsync(m->d_anchor, anchors, (size_t)n * 3 * sizeof(uint32_t),
                            cudaMemcpyHostToDevice, stream));
  {
    std::vector<int32_t> bl;
    bl.reserve((size_t)nb);
    for (int64_t j = 0; j < N; ++j)
      if (m->node_bnd[j]) bl.push_back((int32_t)j);
    CHNS_CUDA(cudaMalloc(&m->d_bnd, std::max<size_t>(bl.size(), 1) * sizeof(int32_t)));
    if (!bl.empty())
      CHNS_CUDA(cudaMemcpyAsync(m->d_bnd, bl.data(), bl.size() * sizeof(int32_t),
                                cudaMemcpyHostToDevice, stream));
    CHNS_CUDA(cudaStreamSynchronize(stream));
  }
  {
    const int64_t np = (int64_t)P.nreg.size();
    m->d.n_patch = np;
    m->n_slots = (int64_t)P.node.size();
    CHNS_CUDA(cudaMalloc(&m->d_patch_elem, (np + 1) * sizeof(int32_t)));
    CHNS_CUDA(cudaMalloc(&m->d_patch_slot, (np + 1) * sizeof(int32_t)));
    CHNS_CUDA(cudaMalloc(&m->d_patch_nreg, np * sizeof(int32_t)));
    CHNS_CUDA(cudaMalloc(&m->d_slot_node, P.node.size() * sizeof(int32_t)));
    CHNS_CUDA(cudaMalloc(&m->d_slot_par, P.par.size() * sizeof(ushort4)));
    CHNS_CUDA(cudaMalloc(&m->d_eloc, (size_t)n * sizeof(uint4)));
    CHNS_CUDA(cudaMemcpy(m->d_patch_elem, P.elem.data(), (np + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    CHNS_CUDA(cudaMemcpy(m->d_patch_slot, P.slot.data(), (np + 1) * sizeof(int32_t), cudaMemcpyHostToDevice));
    CHNS_CUDA(cudaMemcpy(m->d_patch_nreg, P.nreg.data(), np * sizeof(int32_t), cudaMemcpyHostToDevice));
    CHNS_CUDA(cudaMemcpy(m->d_slot_node, P.node.data(), P.node.size() * sizeof(int32_t), cudaMemcpyHostToDevice));
    CHNS_CUDA(cudaMemcpy(m->d_slot_par, P.par.data(), P.par.size() * sizeof(ushort4), cudaMemcpyHostToDevice));
    CHNS_CUDA(cudaMemcpy(m->d_eloc, P.eloc.data(), (size_t)n * sizeof(uint4), cudaMemcpyHostToDevice));
    m->d.patch_elem = m->d_patch_elem;
    m->d.patch_slot = m->d_patch_slot;
    m->d.patch_nreg = m->d_patch_nreg;
    m->d.slot_node = m->d_slot_node;
    m->d.slot_par = m->d_slot_par;
    m->d.eloc = m->d_eloc;
  }
  {
    std::vector<LevelGeo> geo(CHNS_MAXD);
    for (int l = 0; l < CHNS_MAXD; ++l) {
      const double sc = std::ldexp(1.0, -l);
      LevelGeo& G = geo[l];
      for (int d = 0; d < 3; ++d) {
        G.h[d] = extent[d] * sc;
        G.ih[d] = 1.0 / G.h[d];
        G.hf[d] = (float)G.h[d];
        G.ihf[d] = (float)G.ih[d];
      }
      G.detJ = G.h[0] * G.h[1] * G.h[2] * 0.125;
      G.detJf = (float)G.detJ;
    }
    CHNS_CUDA(cudaMalloc(&m->d_geo, CHNS_MAXD * sizeof(LevelGeo)));
    CHNS_CUDA(cudaMemcpy(m->d_geo, geo.data(), CHNS_MAXD * sizeof(LevelGeo), cudaMemcpyHostToDevice));
    m->d.geo = m->d_geo;
  }
  // node coordinates on the device (grid transfer of the learned preconditioner)
  CHNS_CUDA(cudaMalloc(&m->d_node_int, std::max<size_t>(m->node_coords.size(), 3) * sizeof(uint32_t)));
  CHNS_CUDA(cudaMemcpy(m->d_node_int, m->node_coords.data(),
                       m->node_coords.size() * sizeof(uint32_t), cudaMemcpyHostToDevice));
  m->d.enode = m->d_enode;
  m->d.level = m->d_level;
  m->d.hang = m->d_hang;
  m->d.anchor = m->d_anchor;
  int dev = 0;
  CHNS_CUDA(cudaGetDevice(&dev));
  m->device = dev;
  CHNS_CUDA(cudaDeviceGetAttribute(&m->sm_count, cudaDevAttrMultiProcessorCount, dev));
  chns_status st = alloc_workspace(m, light);
  if (st != CHNS_OK) return st;
  CHNS_CUDA(cudaStreamSynchronize(stream));
  return CHNS_OK;
}

}  // namespace chns

extern "C" chns_status chns_mesh_create(const uint32_t* anchors, const uint8_t* levels,
                                        int64_t n_leaves, const double extent[3], void* stream,
                                        chns_mesh** out) {
  if (!anchors || !levels || !extent || !out) {
    chns::set_error("chns_mesh_create: null argument");
    return CHNS_EINVAL;
  }
  *out = nullptr;
  chns_mesh* m = new (std::nothrow) chns_mesh();
  if (!m) {
    chns::set_error("chns_mesh_create: out of host memory");
    return CHNS_ENOMEM;
  }
  chns_status st;
  try {
    st = chns::build_mesh(anchors, levels, n_leaves, extent, chns::as_stream(stream), m, false,
                          false);
  } catch (const std::bad_alloc&) {
    chns::set_error("chns_mesh_create: out of host memory");
    st = CHNS_ENOMEM;
  }
  if (st != CHNS_OK) {
    chns::free_mesh(m);
    return st;
  }
  *out = m;
  return CHNS_OK;
}

extern "C" chns_status chns_mesh_get_info(const chns_mesh* m, chns_mesh_info* info) {
  if (!m || !info) {
    chns::set_error("chns_mesh_get_info: null argument");
    return CHNS_EINVAL;
  }
  info->n_elem = m->d.n_elem;
  info->n_nodes = m->d.n_nodes;
  info->n_hanging = m->d.n_hang;
  info->n_boundary = m->n_boundary;
  info->min_level = m->min_level;
  info->max_level = m->max_level;
  for (int d = 0; d < 3; ++d) info->extent[d] = m->d.ext[d];
  return CHNS_OK;
}

extern "C" chns_status chns_mesh_set_apply_config(chns_mesh* m, chns_apply_kernel kernel,
                                                  int64_t max_ctas) {
  if (!m || max_ctas < 0 || (kernel != CHNS_APPLY_AUTO && kernel != CHNS_APPLY_PATCH &&
                             kernel != CHNS_APPLY_STREAM)) {
    chns::set_error("chns_mesh_set_apply_config: null mesh, unknown kernel or max_ctas < 0");
    return CHNS_EINVAL;
  }
  m->apply_kernel = kernel;
  m->apply_max_ctas = max_ctas;
  return CHNS_OK;
}

extern "C" chns_status chns_mesh_node_coords(const chns_mesh* m, uint32_t* coords) {
  if (!m || !coords) {
    chns::set_error("chns_mesh_node_coords: null argument");
    return CHNS_EINVAL;
  }
  std::memcpy(coords, m->node_coords.data(), m->node_coords.size() * sizeof(uint32_t));
  return CHNS_OK;
}

extern "C" chns_status chns_mesh_boundary(const chns_mesh* m, uint8_t* flags) {
  if (!m || !flags) {
    chns::set_error("chns_mesh_boundary: null argument");
    return CHNS_EINVAL;
  }
  std::memcpy(flags, m->node_bnd.data(), m->node_bnd.size());
  return CHNS_OK;
}

extern "C" void chns_mesh_destroy(chns_mesh* m) { chns::free_mesh(m); }
