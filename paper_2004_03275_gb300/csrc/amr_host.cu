// Host side of the block-tree Euler solver: the quadtree/octree of leaves
// (Morton order, hash lookup), face-neighbour / ghost-slab / reflux tables,
// refine-coarsen decisions with 2:1 balance, CUDA-graph step capture, and the
// amr_* C ABI.
//
// Paper: Sec. 1.3 (block tree, refinement ratio 2, refine when one cell
// exceeds the tolerance, coarsen when every cell is below a fraction of it);
// Sec. 1.2 (CFL step); Sec. 2.3.2 / 2.4 (SSP Runge-Kutta stages).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstddef>
#include <cstdint>
#include <cstring>
#include <memory>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <type_traits>
#include <vector>

#include "../../include/amrvac_gb300.h"
#include "euler_ops.h"
#include "tma.cuh"

using namespace amrgpu;

namespace {

// ------------------------------------------------------------------ tree --
struct LeafH {
  int level;
  int c[3];
};

struct Tree {
  int nd = 2, B = 16, maxlev = 1;
  int base[3] = {1, 1, 1};
  bool periodic[3] = {true, true, true};
  std::vector<LeafH> leaves;
  std::unordered_map<uint64_t, int> index;

  static uint64_t key(int l, const int* c) {
    return ((uint64_t)l << 59) | ((uint64_t)c[0] << 40) | ((uint64_t)c[1] << 20) | (uint64_t)c[2];
  }
  int nblk(int l, int d) const { return d < nd ? base[d] << (l - 1) : 1; }
  int find(int l, const int* c) const {
    if (l < 1 || l > maxlev) return -1;
    for (int d = 0; d < nd; ++d)
      if (c[d] < 0 || c[d] >= nblk(l, d)) return -1;
    auto it = index.find(key(l, c));
    return it == index.end() ? -1 : it->second;
  }
  // wrap block coordinates of level l into the domain; false if outside a non-periodic side
  bool wrap(int l, int* c) const {
    for (int d = 0; d < nd; ++d) {
      int N = nblk(l, d);
      if (c[d] < 0 || c[d] >= N) {
        if (!periodic[d]) return false;
        c[d] = ((c[d] % N) + N) % N;
      }
    }
    return true;
  }
  uint64_t morton(const LeafH& L) const {
    uint64_t X[3] = {0, 0, 0};
    for (int d = 0; d < nd; ++d) X[d] = (uint64_t)L.c[d] << (maxlev - L.level);
    uint64_t k = 0;
    for (int b = 20; b >= 0; --b)
      for (int d = nd - 1; d >= 0; --d) k = (k << 1) | ((X[d] >> b) & 1u);
    return k;
  }
  // sorts leaves by Morton key; returns the permutation new -> old
  std::vector<int> sort_and_index() {
    std::vector<std::pair<uint64_t, int>> ks(leaves.size());
    for (size_t i = 0; i < leaves.size(); ++i) ks[i] = {morton(leaves[i]), (int)i};
    std::sort(ks.begin(), ks.end());
    std::vector<LeafH> sorted(leaves.size());
    std::vector<int> perm(leaves.size());
    for (size_t i = 0; i < ks.size(); ++i) {
      sorted[i] = leaves[ks[i].second];
      perm[i] = ks[i].second;
    }
    leaves.swap(sorted);
    index.clear();
    for (size_t i = 0; i < leaves.size(); ++i) index[key(leaves[i].level, leaves[i].c)] = (int)i;
    return perm;
  }

  // leaves touching block (l, c) (closed boxes, periodic images), excluding the
  // block itself; the block need not be a leaf.  Relies on 2:1 balance only to
  // bound the search depth.
  void cover(int l, const int* n, const int* delta, std::unordered_set<int>& out) const {
    for (int L = l; L >= 1; --L) {
      int a[3] = {0, 0, 0};
      for (int d = 0; d < nd; ++d) a[d] = n[d] >> (l - L);
      int j = find(L, a);
      if (j >= 0) {
        out.insert(j);
        return;
      }
    }
    if (l >= maxlev) return;
    for (int o = 0; o < (1 << nd); ++o) {
      bool ok = true;
      int ch[3] = {0, 0, 0};
      for (int d = 0; d < nd; ++d) {
        int od = (o >> d) & 1;
        if (delta[d] == 1 && od != 0) ok = false;
        if (delta[d] == -1 && od != 1) ok = false;
        ch[d] = 2 * n[d] + od;
      }
      if (ok) cover(l + 1, ch, delta, out);
    }
  }
  void touching(int l, const int* c, std::unordered_set<int>& out, int self) const {
    int tot = 1;
    for (int d = 0; d < nd; ++d) tot *= 3;
    for (int q = 0; q < tot; ++q) {
      int delta[3] = {0, 0, 0}, r = q;
      bool zero = true;
      for (int d = 0; d < nd; ++d) {
        delta[d] = r % 3 - 1;
        r /= 3;
        if (delta[d]) zero = false;
      }
      if (zero) continue;
      int n[3] = {c[0], c[1], c[2]};
      for (int d = 0; d < nd; ++d) n[d] += delta[d];
      if (!wrap(l, n)) continue;
      cover(l, n, delta, out);
    }
    out.erase(self);
  }
};

struct Tables {
  std::vector<int> nb, kind, nbr, ffx;
  std::vector<SlabDesc> slabs;
  std::vector<RefluxRec> rec;  // grouped by coarse leaf, faces ascending within a group
  int nslots = 0;
};

// Face-neighbour codes, ghost slabs at level jumps and reflux records.
bool build_tables(const Tree& T, Tables& tb, std::string* err) {
  const int nd = T.nd, B = T.B, nf = 2 * nd;
  size_t n = T.leaves.size();
  tb.nb.assign(n * nf, -1);
  tb.kind.assign(n * nf, -1);
  tb.nbr.assign(n * nf, -1);
  tb.ffx.assign(n * nf, -1);
  tb.slabs.clear();
  tb.rec.clear();
  tb.nslots = 0;
  auto slot = [&](int leaf, int face) {
    int& s = tb.ffx[(size_t)leaf * nf + face];
    if (s < 0) s = tb.nslots++;
    return s;
  };
  for (size_t i = 0; i < n; ++i) {
    const LeafH& L = T.leaves[i];
    for (int f = 0; f < nf; ++f) {
      int d = f >> 1, side = f & 1;
      int c[3] = {L.c[0], L.c[1], L.c[2]};
      c[d] += side ? 1 : -1;
      size_t o = i * nf + f;
      if (!T.wrap(L.level, c)) continue;  // outflow boundary
      int j = T.find(L.level, c);
      if (j >= 0) {
        tb.nb[o] = j;
        tb.kind[o] = 0;
        tb.nbr[o] = j;
        continue;
      }
      int e1 = -1, e2 = -1;
      for (int e = 0; e < nd; ++e)
        if (e != d) {
          if (e1 < 0) e1 = e; else e2 = e;
        }
      int pc[3] = {c[0] >> 1, c[1] >> 1, c[2] >> 1};
      int jc = L.level > 1 ? T.find(L.level - 1, pc) : -1;
      if (jc >= 0) {
        SlabDesc D{};
        D.target = (int)i;
        D.face = f;
        D.kind = 1;
        D.src[0] = jc;
        D.off[0] = e1 >= 0 ? (L.c[e1] & 1) * (B / 2) : 0;
        D.off[1] = e2 >= 0 ? (L.c[e2] & 1) * (B / 2) : 0;
        tb.nb[o] = -2 - (int)tb.slabs.size();
        tb.slabs.push_back(D);
        tb.kind[o] = 1;
        tb.nbr[o] = jc;
        slot((int)i, f);
        continue;
      }
      // finer neighbours
      SlabDesc D{};
      D.target = (int)i;
      D.face = f;
      D.kind = 0;
      RefluxRec R{};
      R.coarse = (int)i;
      R.face = f;
      int nq = 1 << (nd - 1);
      for (int q = 0; q < nq; ++q) {
        int ch[3] = {0, 0, 0};
        ch[d] = 2 * c[d] + (side ? 0 : 1);
        if (e1 >= 0) ch[e1] = 2 * c[e1] + (q & 1);
        if (e2 >= 0) ch[e2] = 2 * c[e2] + ((q >> 1) & 1);
        int jf = T.find(L.level + 1, ch);
        if (jf < 0) {
          if (err) *err = "tree is not 2:1 balanced or does not cover the domain";
          return false;
        }
        D.src[q] = jf;
        R.fslot[q] = slot(jf, f ^ 1);
      }
      R.cslot = slot((int)i, f);
      tb.nb[o] = -2 - (int)tb.slabs.size();
      tb.slabs.push_back(D);
      tb.rec.push_back(R);
      tb.kind[o] = 2;
      tb.nbr[o] = D.src[0];
    }
  }
  // A coarse cell at a leaf edge or corner may border level jumps in several
  // directions: the records of one coarse leaf form a group (built leaf by leaf,
  // faces ascending) whose corrections a cell receives in that order, x then y then z.
  for (size_t k = 0; k < tb.rec.size();) {
    size_t e = k;
    while (e < tb.rec.size() && tb.rec[e].coarse == tb.rec[k].coarse) ++e;
    for (size_t j = k; j < e; ++j) tb.rec[j].first = (int)k, tb.rec[j].last = (int)e;
    k = e;
  }
  return true;
}

// ------------------------------------------------------------ device buf --
struct DBuf {
  void* p = nullptr;
  size_t cap = 0;
  cudaError_t ensure(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
  }
};

#define CK(call)                                             \
  do {                                                       \
    cudaError_t e_ = (call);                                 \
    if (e_ != cudaSuccess) return h->fail_cuda(e_, #call);   \
  } while (0)

}  // namespace

// ================================================================ handle ==
struct amr_handle {
  amr_config cfg{};
  std::string err;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int nd = 2, B = 16, nv = 4, nc = 256, nt = 16;
  size_t wbytes = 4;
  Tree tree;
  Tables tb;
  Geometry G{};
  // device state
  DBuf U0, Ua, Ub, Unew, stagebuf, partials, gpart, gcount, ctl, nb, level, ffx, slabdesc, slabbuf, rec, fflux, ops,
      errbuf;
  DBuf xyscr;  // float32 3D 16^3: x + y flux differences of the stage (like the state)
  // float32 2D 16^2: TMA tensor maps of the three state buffers viewed as [leaf*4 + var][256]
  CUtensorMap tmaps[3];
  const void* tmap_base[3] = {nullptr, nullptr, nullptr};
  const void* tmap_for(const void* p) const {
    for (int k = 0; k < 3; ++k)
      if (tmap_base[k] == p) return &tmaps[k];
    return nullptr;
  }
  DevCtl* h_ctl = nullptr;  // pinned mirror
  long long steps_seen = 0;
  cudaGraphExec_t graph = nullptr;
  int graph_kernels = 0;
  // float32 2D 16^2 march kernel, per stage kind (first, middle, last): warps per CTA and
  // persistence; chosen by tune_march() before the first captured step unless set by the caller
  int march_tune[3][2] = {{4, 0}, {4, 0}, {4, 1}};
  float march_us[3] = {0.f, 0.f, 0.f};  // time of the chosen launch per stage kind (us)
  bool march_tuned = false;
  long long launches = 0;
  // profiling: when prof_ev is set, events bracket every kernel of a step
  std::vector<cudaEvent_t>* prof_ev = nullptr;  // pairs (before, after)
  std::vector<int>* prof_kind = nullptr;        // 0 stage, 1 ghost fill, 2 reflux, 3 reduce
  void mark_begin() {
    if (!prof_ev) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, stream);
    prof_ev->push_back(e);
  }
  void mark(int kind) {
    if (!prof_ev) return;
    cudaEvent_t e;
    cudaEventCreate(&e);
    cudaEventRecord(e, stream);
    prof_ev->push_back(e);
    prof_kind->push_back(kind);
  }
  int fail(int code, const std::string& m) {
    err = m;
    return code;
  }
  int fail_cuda(cudaError_t e, const char* what) {
    err = std::string("CUDA error ") + cudaGetErrorString(e) + " in " + what;
    return AMR_ERR_CUDA;
  }
  size_t state_bytes(size_t nleaves) const { return nleaves * nv * nc * wbytes; }

  void drop_graph() {
    if (graph) cudaGraphExecDestroy(graph);
    graph = nullptr;
  }

  template <typename real, int ND>
  int dispatch_stage(const StageArgs<real>& a) {
    amr_handle* h = this;
    mark_begin();
    CK((EulerOps<real, ND>::stage(B, cfg.flux, a, G, stream)));
    launches += (std::is_same<real, float>::value && ND == 3 && B == 16) ? 2 : 1;  // 3D: xy and z passes
    mark(0);
    return AMR_OK;
  }

  // ---- the per-precision, per-dimension operations
  template <typename real, int ND>
  int enqueue_step() {
    amr_handle* h = this;
    const int nl = (int)tree.leaves.size();
    const bool jumps = !tb.slabs.empty();
    real* s0 = U0.as<real>();
    real* sa = Ua.as<real>();
    real* sb = Ub.as<real>();
    const int nst = cfg.rk == AMR_SSPRK2 ? 2 : 3;
    const real w2a[2] = {real(0.5), real(0.5)};
    const real w3a[3][2] = {{real(0), real(1)}, {real(0.75), real(0.25)}, {real(1.0 / 3.0), real(2.0 / 3.0)}};
    for (int s = 0; s < nst; ++s) {
      const real* Us = s == 0 ? s0 : (s == 1 ? sa : sb);
      real* out = s == 0 ? sa : (s == 1 ? (nst == 3 ? sb : s0) : s0);
      real alpha = s == 0 ? real(0) : (nst == 2 ? w2a[0] : w3a[s][0]);
      real beta = s == 0 ? real(1) : (nst == 2 ? w2a[1] : w3a[s][1]);
      if (jumps) {
        mark_begin();
        CK((EulerOps<real, ND>::ghost_fill(B, Us, slabbuf.as<real>(), slabdesc.as<SlabDesc>(),
                                           (int)tb.slabs.size(), stream)));
        ++launches;
        mark(1);
      }
      StageArgs<real> a{};
      a.Us = Us;
      a.U0 = s0;
      a.out = out;
      a.nb = nb.as<int>();
      a.slabs = slabbuf.as<real>();
      a.level = level.as<int>();
      a.ffx = ffx.as<int>();
      a.fflux = fflux.as<real>();
      a.scratch = xyscr.as<real>();
      a.tmap_us = tmap_for(Us);
      a.ctl = ctl.as<DevCtl>();
      a.partials = partials.as<double>();
      a.gpart = gpart.as<double>();
      a.gcount = gcount.as<unsigned>();
      a.alpha = alpha;
      a.beta = beta;
      a.stage1 = s == 0;
      a.fuse_reduce = (s == nst - 1) && !jumps;
      a.has_ffx = jumps;
      a.limiter = cfg.limiter;
      a.nleaves = nl;
      {
        const int kind = a.fuse_reduce ? 2 : (a.stage1 ? 0 : 1);
        a.march_nw = march_tune[kind][0];
        a.march_persist = march_tune[kind][1];
      }
      int rc = dispatch_stage<real, ND>(a);
      if (rc) return rc;
      if (jumps) {
        if (!tb.rec.empty()) {
          mark_begin();
          CK((EulerOps<real, ND>::reflux(B, out, fflux.as<real>(), rec.as<RefluxRec>(), (int)tb.rec.size(),
                                         level.as<int>(), G, ctl.as<DevCtl>(), beta, stream)));
          ++launches;
          mark(2);
        }
      }
    }
    if (jumps) {
      mark_begin();
      CK((EulerOps<real, ND>::reduce(B, s0, level.as<int>(), G, ctl.as<DevCtl>(), partials.as<double>(),
                                     gpart.as<double>(), gcount.as<unsigned>(), nl, 1, stream)));
      ++launches;
      mark(3);
    }
    return AMR_OK;
  }

  template <typename real, int ND>
  int ghost_fill_current(const real* U) {
    amr_handle* h = this;
    if (tb.slabs.empty()) return AMR_OK;
    CK((EulerOps<real, ND>::ghost_fill(B, U, slabbuf.as<real>(), slabdesc.as<SlabDesc>(), (int)tb.slabs.size(),
                                       stream)));
    ++launches;
    return AMR_OK;
  }

  int run_typed(const char* what);
};

namespace {

template <typename F>
int with_type(amr_handle* h, F&& f) {
  if (h->cfg.precision == AMR_FP64) {
    switch (h->nd) {
      case 1: return f.template operator()<double, 1>();
      case 2: return f.template operator()<double, 2>();
      default: return f.template operator()<double, 3>();
    }
  }
  switch (h->nd) {
    case 1: return f.template operator()<float, 1>();
    case 2: return f.template operator()<float, 2>();
    default: return f.template operator()<float, 3>();
  }
}

int upload_tables(amr_handle* h) {
  auto& tb = h->tb;
  auto& T = h->tree;
  size_t n = T.leaves.size();
  int nf = 2 * h->nd;
  std::vector<int> lev(n);
  for (size_t i = 0; i < n; ++i) lev[i] = T.leaves[i].level;
#define CKH(call)                                               \
  do {                                                          \
    cudaError_t e_ = (call);                                    \
    if (e_ != cudaSuccess) return h->fail_cuda(e_, #call);      \
  } while (0)
  CKH(h->nb.ensure(std::max<size_t>(1, n * nf) * sizeof(int)));
  CKH(h->ffx.ensure(std::max<size_t>(1, n * nf) * sizeof(int)));
  CKH(h->level.ensure(std::max<size_t>(1, n) * sizeof(int)));
  CKH(h->slabdesc.ensure(std::max<size_t>(1, tb.slabs.size()) * sizeof(SlabDesc)));
  CKH(h->slabbuf.ensure(std::max<size_t>(1, tb.slabs.size()) * h->nv * 2 * h->nt * h->wbytes));
  CKH(h->rec.ensure(std::max<size_t>(1, tb.rec.size()) * sizeof(RefluxRec)));
  CKH(h->fflux.ensure(std::max<size_t>(1, (size_t)tb.nslots) * h->nv * h->nt * h->wbytes));
  // one partial per leaf, or per CTA of a stage kernel (up to 4 CTAs per leaf)
  CKH(h->partials.ensure(std::max<size_t>(1, 4 * n) * h->nv * sizeof(double)));
  CKH(h->errbuf.ensure(std::max<size_t>(1, n) * sizeof(double)));
  CKH(cudaMemcpyAsync(h->nb.p, tb.nb.data(), n * nf * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CKH(cudaMemcpyAsync(h->ffx.p, tb.ffx.data(), n * nf * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  CKH(cudaMemcpyAsync(h->level.p, lev.data(), n * sizeof(int), cudaMemcpyHostToDevice, h->stream));
  if (!tb.slabs.empty())
    CKH(cudaMemcpyAsync(h->slabdesc.p, tb.slabs.data(), tb.slabs.size() * sizeof(SlabDesc), cudaMemcpyHostToDevice,
                        h->stream));
  if (!tb.rec.empty())
    CKH(cudaMemcpyAsync(h->rec.p, tb.rec.data(), tb.rec.size() * sizeof(RefluxRec), cudaMemcpyHostToDevice,
                        h->stream));
  CKH(cudaStreamSynchronize(h->stream));
  h->G.nleaves = (int)n;
  if (h->nd == 2 && h->B == 16 && h->wbytes == 4 && n > 0) {
    const DBuf* bufs[3] = {&h->U0, &h->Ua, &h->Ub};
    for (int k = 0; k < 3; ++k) {
      CKH(encode_tmap_2d(&h->tmaps[k], bufs[k]->as<float>(), (uint64_t)n * 4, 256, 256, 4));
      h->tmap_base[k] = bufs[k]->p;
    }
  }
  h->drop_graph();
  return AMR_OK;
}

int rebuild(amr_handle* h) {
  std::string e;
  if (!build_tables(h->tree, h->tb, &e)) return h->fail(AMR_ERR_UNBALANCED, e);
  return upload_tables(h);
}

// recompute dt_cfl and totals of the current state (no time advance)
int refresh_reduce(amr_handle* h) {
  int nl = (int)h->tree.leaves.size();
  return with_type(h, [&]<typename real, int ND>() -> int {
    cudaError_t e = EulerOps<real, ND>::reduce(h->B, h->U0.as<real>(), h->level.as<int>(), h->G,
                                               h->ctl.as<DevCtl>(), h->partials.as<double>(), h->gpart.as<double>(),
                                               h->gcount.as<unsigned>(), nl, 0, h->stream);
    if (e != cudaSuccess) return h->fail_cuda(e, "reduce");
    ++h->launches;
    return AMR_OK;
  });
}

int sync_ctl(amr_handle* h) {
  CKH(cudaMemcpyAsync(h->h_ctl, h->ctl.p, sizeof(DevCtl), cudaMemcpyDeviceToHost, h->stream));
  CKH(cudaStreamSynchronize(h->stream));
  if (h->h_ctl->status & 2) return h->fail(AMR_ERR_TIMEOUT, "a bounded wait for a TMA copy gave up");
  if (h->h_ctl->status & 1) return h->fail(AMR_ERR_NONPHYSICAL, "non-positive density or pressure met");
  return AMR_OK;
}

bool balanced_cover(const Tree& T, std::string* err) {
  // volume check + pairwise 2:1 check through touching()
  long double vol = 0, tot = 1;
  for (int d = 0; d < T.nd; ++d) tot *= (long double)T.base[d] * (1 << (T.maxlev - 1));
  for (auto& L : T.leaves) {
    long double v = 1;
    for (int d = 0; d < T.nd; ++d) v *= (long double)(1 << (T.maxlev - L.level));
    vol += v;
  }
  if (vol != tot) {
    *err = "leaves do not cover the domain exactly";
    return false;
  }
  for (size_t i = 0; i < T.leaves.size(); ++i) {
    std::unordered_set<int> t;
    T.touching(T.leaves[i].level, T.leaves[i].c, t, (int)i);
    for (int j : t)
      if (std::abs(T.leaves[j].level - T.leaves[i].level) > 1) {
        *err = "leaves are not 2:1 balanced";
        return false;
      }
  }
  return true;
}

}  // namespace

// ================================================================== ABI ==
extern "C" {

int amr_create(const amr_config* cfg, amr_handle** out) {
  if (!cfg || !out) return AMR_ERR_INVALID_ARG;
  *out = nullptr;
  if (cfg->ndim < 1 || cfg->ndim > 3) return AMR_ERR_INVALID_ARG;
  if (cfg->block_nx != 8 && cfg->block_nx != 16) return AMR_ERR_INVALID_ARG;
  if (cfg->max_level < 1 || cfg->max_level > kMaxLevel) return AMR_ERR_INVALID_ARG;
  if (cfg->flux < 0 || cfg->flux > 2 || cfg->limiter < 0 || cfg->limiter > 5) return AMR_ERR_INVALID_ARG;
  if (cfg->rk != AMR_SSPRK2 && cfg->rk != AMR_SSPRK3) return AMR_ERR_INVALID_ARG;
  if (cfg->precision != AMR_FP64 && cfg->precision != AMR_FP32) return AMR_ERR_INVALID_ARG;
  if (!(cfg->gamma > 1.0) || !(cfg->cfl > 0.0)) return AMR_ERR_INVALID_ARG;
  long long nbase = 1;
  for (int d = 0; d < cfg->ndim; ++d) {
    if (cfg->base_nblocks[d] < 1 || !(cfg->xmax[d] > cfg->xmin[d])) return AMR_ERR_INVALID_ARG;
    if ((long long)cfg->base_nblocks[d] << (cfg->max_level - 1) >= (1LL << 19)) return AMR_ERR_INVALID_ARG;
    if ((cfg->bc[d][0] == AMR_BC_PERIODIC) != (cfg->bc[d][1] == AMR_BC_PERIODIC)) return AMR_ERR_INVALID_ARG;
    nbase *= cfg->base_nblocks[d];
  }
  if (cfg->max_blocks < nbase) return AMR_ERR_CAPACITY;
  std::unique_ptr<amr_handle> h(new amr_handle());
  h->cfg = *cfg;
  h->stream = (cudaStream_t)cfg->stream;
  if (!h->stream) {  // graph capture needs a non-legacy stream
    if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess) return AMR_ERR_CUDA;
    h->own_stream = true;
  }
  h->nd = cfg->ndim;
  h->B = cfg->block_nx;
  h->nv = cfg->ndim + 2;
  h->nc = 1;
  for (int d = 0; d < h->nd; ++d) h->nc *= h->B;
  h->nt = h->nc / h->B;
  h->wbytes = cfg->precision == AMR_FP64 ? 8 : 4;
  Tree& T = h->tree;
  T.nd = h->nd;
  T.B = h->B;
  T.maxlev = cfg->max_level;
  for (int d = 0; d < 3; ++d) {
    T.base[d] = d < h->nd ? cfg->base_nblocks[d] : 1;
    T.periodic[d] = d < h->nd ? cfg->bc[d][0] == AMR_BC_PERIODIC : true;
  }
  for (int z = 0; z < T.nblk(1, 2); ++z)
    for (int y = 0; y < T.nblk(1, 1); ++y)
      for (int x = 0; x < T.nblk(1, 0); ++x) T.leaves.push_back(LeafH{1, {x, y, z}});
  T.sort_and_index();
  // geometry
  Geometry& G = h->G;
  G.ndim = h->nd;
  G.bnx = h->B;
  G.gamma = cfg->gamma;
  G.cfl = cfg->cfl;
  for (int l = 1; l <= kMaxLevel; ++l) {
    double dV = 1.0;
    for (int d = 0; d < 3; ++d) {
      double n = d < h->nd ? (double)cfg->base_nblocks[d] * h->B * (double)(1LL << (l - 1)) : 1.0;
      G.dx[l][d] = d < h->nd ? (cfg->xmax[d] - cfg->xmin[d]) / n : 1.0;
      if (d < h->nd) dV = dV * G.dx[l][d];
    }
    G.dV[l] = dV;
    for (int d = 0; d < 3; ++d) {
      G.dxf[l][d] = (float)G.dx[l][d];
      G.idxf[l][d] = (float)(1.0 / G.dx[l][d]);
    }
  }
  G.gammaf = (float)cfg->gamma;
  size_t sb = h->state_bytes((size_t)cfg->max_blocks);
  cudaError_t e;
  if ((e = h->U0.ensure(sb)) != cudaSuccess || (e = h->Ua.ensure(sb)) != cudaSuccess ||
      (e = h->Ub.ensure(sb)) != cudaSuccess || (e = h->ctl.ensure(sizeof(DevCtl))) != cudaSuccess ||
      (e = h->gpart.ensure((4 * (size_t)cfg->max_blocks / kGroupCTAs + 2) * 5 * sizeof(double))) != cudaSuccess ||
      (e = h->gcount.ensure((4 * (size_t)cfg->max_blocks / kGroupCTAs + 2) * sizeof(unsigned))) != cudaSuccess ||
      (h->nd == 3 && h->B == 16 && h->wbytes == 4 && (e = h->xyscr.ensure(sb)) != cudaSuccess) ||
      (e = cudaMallocHost(&h->h_ctl, sizeof(DevCtl))) != cudaSuccess)
    return e == cudaErrorMemoryAllocation ? AMR_ERR_OOM : AMR_ERR_CUDA;
  DevCtl c0{};
  c0.cfl = cfg->cfl;
  c0.t_end = 1e300;
  if (cudaMemcpy(h->ctl.p, &c0, sizeof(DevCtl), cudaMemcpyHostToDevice) != cudaSuccess) return AMR_ERR_CUDA;
  if (cudaMemset(h->U0.p, 0, h->state_bytes(T.leaves.size())) != cudaSuccess) return AMR_ERR_CUDA;
  if (cudaMemset(h->gcount.p, 0, h->gcount.cap) != cudaSuccess) return AMR_ERR_CUDA;
  int rc = rebuild(h.get());
  if (rc) return rc;
  amr_handle* hp = h.get();
  rc = with_type(hp, [&]<typename real, int ND>() -> int {
    cudaError_t e2 = EulerOps<real, ND>::prepare(hp->B, hp->cfg.flux, hp->cfg.limiter);
    return e2 == cudaSuccess ? AMR_OK : hp->fail_cuda(e2, "prepare");
  });
  if (rc) return rc;
  *out = h.release();
  return AMR_OK;
}

int amr_destroy(amr_handle* h) {
  if (!h) return AMR_ERR_INVALID_ARG;
  h->drop_graph();
  for (DBuf* b : {&h->xyscr, &h->U0, &h->Ua, &h->Ub, &h->Unew, &h->stagebuf, &h->partials, &h->gpart, &h->gcount, &h->ctl, &h->nb, &h->level,
                  &h->ffx, &h->slabdesc, &h->slabbuf, &h->rec, &h->fflux, &h->ops, &h->errbuf})
    b->release();
  if (h->h_ctl) cudaFreeHost(h->h_ctl);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
  return AMR_OK;
}

const char* amr_last_error(const amr_handle* h) { return h ? h->err.c_str() : "null handle"; }

int amr_num_leaves(const amr_handle* h, long long* n) {
  if (!h || !n) return AMR_ERR_INVALID_ARG;
  *n = (long long)h->tree.leaves.size();
  return AMR_OK;
}

int amr_leaf_info(const amr_handle* h, int* level, int* coords, long long cap) {
  if (!h || cap < (long long)h->tree.leaves.size()) return AMR_ERR_INVALID_ARG;
  for (size_t i = 0; i < h->tree.leaves.size(); ++i) {
    if (level) level[i] = h->tree.leaves[i].level;
    if (coords)
      for (int d = 0; d < 3; ++d) coords[3 * i + d] = h->tree.leaves[i].c[d];
  }
  return AMR_OK;
}

int amr_set_leaves(amr_handle* h, long long n, const int* level, const int* coords) {
  if (!h || n < 1 || !level || !coords) return AMR_ERR_INVALID_ARG;
  if (n > h->cfg.max_blocks) return h->fail(AMR_ERR_CAPACITY, "more leaves than max_blocks");
  Tree T = h->tree;
  T.leaves.clear();
  for (long long i = 0; i < n; ++i) {
    LeafH L{level[i], {coords[3 * i], coords[3 * i + 1], coords[3 * i + 2]}};
    if (L.level < 1 || L.level > T.maxlev) return h->fail(AMR_ERR_INVALID_ARG, "leaf level out of range");
    for (int d = 0; d < 3; ++d) {
      if (d >= T.nd) L.c[d] = 0;
      else if (L.c[d] < 0 || L.c[d] >= T.nblk(L.level, d)) return h->fail(AMR_ERR_INVALID_ARG, "leaf outside domain");
    }
    T.leaves.push_back(L);
  }
  T.sort_and_index();
  if (T.index.size() != T.leaves.size()) return h->fail(AMR_ERR_UNBALANCED, "duplicate leaves");
  std::string e;
  if (!balanced_cover(T, &e)) return h->fail(AMR_ERR_UNBALANCED, e);
  h->tree = T;
  int rc = rebuild(h);
  if (rc) return rc;
  CK(cudaMemsetAsync(h->U0.p, 0, h->state_bytes(n), h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return AMR_OK;
}

// Device address of page-locked (pinned) host memory, which kernels read and write in place
// (zero copy: one pass over the host buffer instead of a copy engine pass plus a pass over a
// staging buffer); nullptr for pageable memory.
static const void* pinned_device_ptr(const void* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int amr_set_state(amr_handle* h, const double* W, long long n_values, int on_device, int primitive) {
  if (!h || !W) return AMR_ERR_INVALID_ARG;
  long long nl = (long long)h->tree.leaves.size();
  long long need = nl * h->nv * h->nc;
  if (n_values != need) return h->fail(AMR_ERR_INVALID_ARG, "n_values does not match leaves*(ndim+2)*cells");
  // the conversion kernel reads two doubles per 16-byte load: an array that is not 16-byte
  // aligned, or pageable host memory, goes through the (aligned) staging buffer
  const double* src = W;
  const void* pin = on_device ? nullptr : pinned_device_ptr(W);
  if (pin) src = static_cast<const double*>(pin);
  if ((!on_device && !pin) || (reinterpret_cast<uintptr_t>(src) & 15)) {
    CK(h->stagebuf.ensure(need * sizeof(double)));
    CK(cudaMemcpyAsync(h->stagebuf.p, W, need * sizeof(double), cudaMemcpyDefault, h->stream));
    src = h->stagebuf.as<double>();
  }
  int rc = with_type(h, [&]<typename real, int ND>() -> int {
    cudaError_t e = EulerOps<real, ND>::set_state(h->B, src, h->U0.as<real>(), nl, primitive, h->cfg.gamma, h->stream);
    if (e != cudaSuccess) return h->fail_cuda(e, "set_state");
    ++h->launches;
    return AMR_OK;
  });
  if (rc) return rc;
  // clear the status word, then recompute dt and totals
  CK(cudaMemsetAsync((char*)h->ctl.p + offsetof(DevCtl, status), 0, sizeof(int), h->stream));
  rc = refresh_reduce(h);
  if (rc) return rc;
  return sync_ctl(h);
}

int amr_read_state(amr_handle* h, double* U, long long cap_values, int on_device) {
  if (!h || !U) return AMR_ERR_INVALID_ARG;
  long long nl = (long long)h->tree.leaves.size();
  long long need = nl * h->nv * h->nc;
  if (cap_values < need) return h->fail(AMR_ERR_INVALID_ARG, "output buffer too small");
  // pageable host memory is written through the staging buffer
  double* dst = U;
  bool staged = false;
  const void* pin = on_device ? nullptr : pinned_device_ptr(U);
  if (pin) dst = static_cast<double*>(const_cast<void*>(pin));
  if (!on_device && !pin) {
    CK(h->stagebuf.ensure(need * sizeof(double)));
    dst = h->stagebuf.as<double>();
    staged = true;
  }
  int rc = with_type(h, [&]<typename real, int ND>() -> int {
    cudaError_t e = EulerOps<real, ND>::read_state(h->U0.as<real>(), dst, need, h->stream);
    if (e != cudaSuccess) return h->fail_cuda(e, "read_state");
    ++h->launches;
    return AMR_OK;
  });
  if (rc) return rc;
  if (staged) CK(cudaMemcpyAsync(U, dst, need * sizeof(double), cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return AMR_OK;
}

int amr_set_time(amr_handle* h, double t) {
  if (!h) return AMR_ERR_INVALID_ARG;
  CK(ctl_set_t(h->ctl.as<DevCtl>(), t, h->stream));
  ++h->launches;
  CK(cudaStreamSynchronize(h->stream));
  return AMR_OK;
}

static int capture_graph(amr_handle* h) {
  cudaGraph_t g;
  CK(cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal));
  long long before = h->launches;
  int rc = with_type(h, [&]<typename real, int ND>() -> int { return h->enqueue_step<real, ND>(); });
  cudaError_t ec = cudaStreamEndCapture(h->stream, &g);
  if (rc) return rc;
  if (ec != cudaSuccess) return h->fail_cuda(ec, "cudaStreamEndCapture");
  h->graph_kernels = (int)(h->launches - before);
  h->launches = before;
  cudaError_t ei = cudaGraphInstantiate(&h->graph, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    h->graph = nullptr;
    return h->fail_cuda(ei, "cudaGraphInstantiate");
  }
  return AMR_OK;
}

// Stage-kernel tuner (float32 2D 16^2 leaves, uniform grids, SSPRK3).  Candidates per stage
// kind: warps (leaves) per CTA in {2, 4, 8} and grid or persistent launch for the first and
// middle stages, grid or persistent launch for the last stage (its CTAs have 4 warps).  The
// kinds are tuned in turn, the others at their current choice: each candidate's step is
// captured as the run's graph would be and replayed kTuneWarm times untimed and kTuneSteps times timed,
// in kTuneRounds rounds over the candidates (best round kept)
// (CUDA events around the replays, so every stage sees the cache state and launch sequence
// of a real step), from a saved copy of the state and control block that is put back after
// every candidate and at the end, so that neither the state nor the time advances.  Every candidate computes the same state bit for bit (tested); the fastest step
// is kept.  Runs once, before the first captured step.
constexpr int kTuneSteps = 10;
constexpr int kTuneRounds = 3;
constexpr int kTuneWarm = 5;

static int tune_march(amr_handle* h) {
  h->march_tuned = true;
  if (h->cfg.precision != AMR_FP32 || h->nd != 2 || h->B != 16 || !h->tb.slabs.empty() ||
      h->tree.leaves.empty() || h->cfg.rk != AMR_SSPRK3)
    return AMR_OK;
  const size_t sb = h->state_bytes(h->tree.leaves.size());
  DBuf keepU, keepC;
  CK(keepU.ensure(sb));
  CK(keepC.ensure(sizeof(DevCtl)));
  CK(cudaMemcpyAsync(keepU.p, h->U0.p, sb, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemcpyAsync(keepC.p, h->ctl.p, sizeof(DevCtl), cudaMemcpyDeviceToDevice, h->stream));
  auto restore = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(h->U0.p, keepU.p, sb, cudaMemcpyDeviceToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(h->ctl.p, keepC.p, sizeof(DevCtl), cudaMemcpyDeviceToDevice, h->stream);
    return e;
  };
  CK(ctl_set_t_end(h->ctl.as<DevCtl>(), 1e300, h->stream));  // no end-time clip while timing (restored after)
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  int rc = AMR_OK;
  static const int cands[2][6][2] = {{{4, 0}, {2, 0}, {8, 0}, {4, 1}, {2, 1}, {8, 1}},
                                     {{4, 1}, {4, 0}, {0, 0}, {0, 0}, {0, 0}, {0, 0}}};
  for (int k = 0; k < 3 && !rc; ++k) {
    const int nc = k < 2 ? 6 : 2;
    // one captured step per candidate, then kTuneRounds rounds over the candidates in turn (so
    // that clock ramps and cache history spread over all of them); a candidate's time is its
    // best round
    cudaGraphExec_t gx[6] = {};
    float best[6];
    for (int c = 0; c < nc; ++c) best[c] = 1e30f;
    for (int c = 0; c < nc && !rc; ++c) {
      h->march_tune[k][0] = cands[k < 2 ? 0 : 1][c][0];
      h->march_tune[k][1] = cands[k < 2 ? 0 : 1][c][1];
      h->drop_graph();
      rc = capture_graph(h);
      gx[c] = h->graph;
      h->graph = nullptr;
    }
    for (int round = 0; round < kTuneRounds && !rc; ++round)
      for (int c = 0; c < nc && !rc; ++c) {
        // warm-up steps: the restore leaves the whole state in L2, which a real run's stages
        // do not see; a few steps bring the cache back to its running state
        cudaError_t e = cudaSuccess;
        for (int r = 0; r < kTuneWarm && e == cudaSuccess; ++r) e = cudaGraphLaunch(gx[c], h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
        for (int r = 0; r < kTuneSteps && e == cudaSuccess; ++r) e = cudaGraphLaunch(gx[c], h->stream);
        if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
        if (e == cudaSuccess) e = restore();
        if (e == cudaSuccess) e = ctl_set_t_end(h->ctl.as<DevCtl>(), 1e300, h->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) {
          rc = h->fail_cuda(e, "stage tuner");
          break;
        }
        best[c] = std::min(best[c], ms);
      }
    for (int c = 0; c < nc; ++c)
      if (gx[c]) cudaGraphExecDestroy(gx[c]);
    int bc = 0;
    for (int c = 1; c < nc; ++c)
      if (best[c] < best[bc]) bc = c;
    h->march_tune[k][0] = cands[k < 2 ? 0 : 1][bc][0];
    h->march_tune[k][1] = cands[k < 2 ? 0 : 1][bc][1];
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->drop_graph();  // the caller captures the step with the chosen launches
  if (rc) {
    restore();
    return rc;
  }
  CK(restore());
  CK(ctl_set_t_end(h->ctl.as<DevCtl>(), 1e300, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  // the chosen launches' own times, from one profiled step of the restored state
  std::vector<cudaEvent_t> ev;
  std::vector<int> kinds;
  h->prof_ev = &ev;
  h->prof_kind = &kinds;
  rc = h->enqueue_step<float, 2>();
  h->prof_ev = nullptr;
  h->prof_kind = nullptr;
  cudaError_t e = rc ? cudaSuccess : cudaStreamSynchronize(h->stream);
  for (size_t i = 0; e == cudaSuccess && i + 1 < ev.size() && i / 2 < 3; i += 2) {
    float ms = 0.f;
    e = cudaEventElapsedTime(&ms, ev[i], ev[i + 1]);
    h->march_us[i / 2] = ms * 1e3f;
  }
  for (cudaEvent_t x : ev) cudaEventDestroy(x);
  if (!rc && e != cudaSuccess) rc = h->fail_cuda(e, "stage tuner events");
  if (!rc) CK(restore());
  if (!rc) CK(cudaStreamSynchronize(h->stream));
  return rc;
}

static int ensure_graph(amr_handle* h) {
  if (h->graph) return AMR_OK;
  if (!h->march_tuned)
    if (int rc = tune_march(h)) return rc;
  return capture_graph(h);
}

int amr_run(amr_handle* h, int nsteps, double t_end) {
  if (!h || nsteps < 0) return AMR_ERR_INVALID_ARG;
  int rc = ensure_graph(h);
  if (rc) return rc;
  CK(ctl_set_t_end(h->ctl.as<DevCtl>(), t_end, h->stream));
  ++h->launches;
  for (int i = 0; i < nsteps; ++i) {
    CK(cudaGraphLaunch(h->graph, h->stream));
    h->launches += h->graph_kernels;
  }
  return AMR_OK;
}

int amr_sync(amr_handle* h, double* t_now, double* dt_last) {
  if (!h) return AMR_ERR_INVALID_ARG;
  int rc = sync_ctl(h);
  if (t_now) *t_now = h->h_ctl->t;
  if (dt_last) *dt_last = h->h_ctl->dt_last;
  h->steps_seen = h->h_ctl->steps;
  return rc;
}

int amr_step(amr_handle* h, double t_end, double* dt_taken, double* t_now) {
  if (!h) return AMR_ERR_INVALID_ARG;
  long long before = h->steps_seen;
  int rc = amr_run(h, 1, t_end);
  if (rc) return rc;
  double t, dtl;
  rc = amr_sync(h, &t, &dtl);
  if (t_now) *t_now = t;
  if (dt_taken) *dt_taken = h->steps_seen > before ? dtl : 0.0;
  return rc;
}

int amr_conserved_totals(amr_handle* h, double* totals) {
  if (!h || !totals) return AMR_ERR_INVALID_ARG;
  int rc = sync_ctl(h);
  for (int v = 0; v < h->nv; ++v) totals[v] = h->h_ctl->totals[v];
  return rc;
}

int amr_estimate(amr_handle* h, double* err, long long cap) {
  long long nl = h ? (long long)h->tree.leaves.size() : 0;
  if (!h || !err || cap < nl) return AMR_ERR_INVALID_ARG;
  int rc = with_type(h, [&]<typename real, int ND>() -> int {
    int r = h->ghost_fill_current<real, ND>(h->U0.as<real>());
    if (r) return r;
    cudaError_t e = EulerOps<real, ND>::lohner(h->B, h->U0.as<real>(), h->slabbuf.as<real>(), h->nb.as<int>(),
                                               h->cfg.gamma, h->cfg.wavefilter, h->cfg.refine_var_mask,
                                               h->errbuf.as<double>(), (int)nl, h->stream);
    if (e != cudaSuccess) return h->fail_cuda(e, "lohner");
    ++h->launches;
    return AMR_OK;
  });
  if (rc) return rc;
  CK(cudaMemcpyAsync(err, h->errbuf.p, nl * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return AMR_OK;
}

// Refine / coarsen with 2:1 balance (Sec. 1.3); see the header for the rules.
int amr_regrid(amr_handle* h) {
  if (!h) return AMR_ERR_INVALID_ARG;
  Tree& T = h->tree;
  const int nd = T.nd;
  size_t nl = T.leaves.size();
  std::vector<double> err(nl);
  int rc = amr_estimate(h, err.data(), (long long)nl);
  if (rc) return rc;
  std::vector<char> ref(nl, 0), crs(nl, 0);
  for (size_t i = 0; i < nl; ++i) {
    int lev = T.leaves[i].level;
    if (lev < T.maxlev && err[i] > h->cfg.refine_tol) ref[i] = 1;
    if (lev > 1 && err[i] < h->cfg.coarsen_frac * h->cfg.refine_tol) crs[i] = 1;
  }
  // refinement closes over coarser touching leaves
  std::vector<int> work;
  for (size_t i = 0; i < nl; ++i)
    if (ref[i]) work.push_back((int)i);
  while (!work.empty()) {
    int i = work.back();
    work.pop_back();
    std::unordered_set<int> t;
    T.touching(T.leaves[i].level, T.leaves[i].c, t, i);
    for (int j : t)
      if (!ref[j] && T.leaves[j].level < T.leaves[i].level) {
        ref[j] = 1;
        work.push_back(j);
      }
  }
  // coarsening groups
  int nch = 1 << nd;
  std::vector<char> merged(nl, 0);
  std::vector<std::vector<int>> groups;
  for (size_t i = 0; i < nl; ++i) {
    const LeafH& A = T.leaves[i];
    if (A.level == 1) continue;
    bool first = true;
    for (int d = 0; d < nd; ++d)
      if (A.c[d] & 1) first = false;
    if (!first) continue;
    std::vector<int> kids;
    bool ok = true;
    for (int o = 0; o < nch && ok; ++o) {
      int c[3] = {A.c[0] + (o & 1), nd > 1 ? A.c[1] + ((o >> 1) & 1) : 0, nd > 2 ? A.c[2] + ((o >> 2) & 1) : 0};
      int j = T.find(A.level, c);
      if (j < 0 || ref[j] || !crs[j]) ok = false;
      kids.push_back(j);
    }
    if (!ok) continue;
    int pc[3] = {A.c[0] >> 1, A.c[1] >> 1, A.c[2] >> 1};
    std::unordered_set<int> t;
    T.touching(A.level - 1, pc, t, -1);
    for (int j : t)
      if (T.leaves[j].level + (ref[j] ? 1 : 0) > A.level) ok = false;
    if (!ok) continue;
    for (int k : kids) merged[k] = 1;
    groups.push_back(kids);
  }
  // new leaves and the ops that fill them
  Tree NT = T;
  NT.leaves.clear();
  std::vector<RegridOp> ops;
  for (size_t i = 0; i < nl; ++i) {
    const LeafH& L = T.leaves[i];
    if (ref[i]) {
      for (int o = 0; o < nch; ++o) {
        LeafH C{L.level + 1, {0, 0, 0}};
        for (int d = 0; d < nd; ++d) C.c[d] = 2 * L.c[d] + ((o >> d) & 1);
        NT.leaves.push_back(C);
        RegridOp op{};
        op.kind = 1;
        op.src[0] = (int)i;
        op.child = o;
        ops.push_back(op);
      }
    } else if (!merged[i]) {
      NT.leaves.push_back(L);
      RegridOp op{};
      op.kind = 0;
      op.src[0] = (int)i;
      ops.push_back(op);
    }
  }
  for (auto& g : groups) {
    const LeafH& A = T.leaves[g[0]];
    LeafH P{A.level - 1, {A.c[0] >> 1, A.c[1] >> 1, A.c[2] >> 1}};
    NT.leaves.push_back(P);
    RegridOp op{};
    op.kind = 2;
    for (int o = 0; o < nch; ++o) op.src[o] = g[o];
    ops.push_back(op);
  }
  if ((long long)NT.leaves.size() > h->cfg.max_blocks)
    return h->fail(AMR_ERR_CAPACITY, "regrid would exceed max_blocks");
  std::vector<int> perm = NT.sort_and_index();
  std::vector<RegridOp> sops(ops.size());
  for (size_t i = 0; i < perm.size(); ++i) sops[i] = ops[perm[i]];
  // device: ghosts of the old tree (parents' edge slopes), then build the new state
  CK(h->ops.ensure(std::max<size_t>(1, sops.size()) * sizeof(RegridOp)));
  CK(cudaMemcpyAsync(h->ops.p, sops.data(), sops.size() * sizeof(RegridOp), cudaMemcpyHostToDevice, h->stream));
  rc = with_type(h, [&]<typename real, int ND>() -> int {
    int r = h->ghost_fill_current<real, ND>(h->U0.as<real>());
    if (r) return r;
    cudaError_t e = EulerOps<real, ND>::regrid(h->B, h->U0.as<real>(), h->Ua.as<real>(), h->slabbuf.as<real>(),
                                               h->nb.as<int>(), h->ops.as<RegridOp>(), (int)sops.size(), h->stream);
    if (e != cudaSuccess) return h->fail_cuda(e, "regrid");
    ++h->launches;
    return AMR_OK;
  });
  if (rc) return rc;
  CK(cudaStreamSynchronize(h->stream));
  std::swap(h->U0, h->Ua);
  h->tree = NT;
  rc = rebuild(h);
  if (rc) return rc;
  rc = refresh_reduce(h);
  if (rc) return rc;
  return sync_ctl(h);
}

int amr_set_state_fn(amr_handle* h, amr_prim_fn prim_at, void* user) {
  if (!h || !prim_at) return AMR_ERR_INVALID_ARG;
  const int nd = h->nd, B = h->B, nv = h->nv, nc = h->nc;
  const int passes = std::max(1, h->cfg.max_level);
  std::vector<double> W, V(nv);
  for (int pass = 0; pass < passes; ++pass) {
    if (pass > 0) {
      int rc = amr_regrid(h);  // refine where the sampled state asks for it, then resample
      if (rc) return rc;
    }
    const size_t nl = h->tree.leaves.size();
    W.assign(nl * nv * nc, 0.0);
    for (size_t l = 0; l < nl; ++l) {
      const LeafH& L = h->tree.leaves[l];
      double dx[3] = {0.0, 0.0, 0.0};
      for (int d = 0; d < nd; ++d) {
        const double cells = (double)h->cfg.base_nblocks[d] * B * (double)(1ll << (L.level - 1));
        dx[d] = (h->cfg.xmax[d] - h->cfg.xmin[d]) / cells;
      }
      for (int cell = 0; cell < nc; ++cell) {
        const int loc[3] = {cell % B, nd > 1 ? (cell / B) % B : 0, nd > 2 ? cell / (B * B) : 0};
        double x[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < nd; ++d) {
          const double g = (double)L.c[d] * B + loc[d];  // global cell index on the leaf's level
          x[d] = h->cfg.xmin[d] + (g + 0.5) * dx[d];
        }
        prim_at(x, V.data(), user);
        for (int v = 0; v < nv; ++v) W[(l * nv + v) * nc + cell] = V[v];
      }
    }
    int rc = amr_set_state(h, W.data(), (long long)W.size(), 0, 1);
    if (rc) return rc;
  }
  return AMR_OK;
}

int amr_face_neighbors(const amr_handle* h, int* kind, int* nbr, long long cap) {
  if (!h) return AMR_ERR_INVALID_ARG;
  size_t n = h->tb.kind.size();
  if (cap < (long long)n) return AMR_ERR_INVALID_ARG;
  if (kind) std::memcpy(kind, h->tb.kind.data(), n * sizeof(int));
  if (nbr) std::memcpy(nbr, h->tb.nbr.data(), n * sizeof(int));
  return AMR_OK;
}

int amr_face_ghosts(amr_handle* h, long long leaf, double* out, long long cap) {
  if (!h || !out || leaf < 0 || leaf >= (long long)h->tree.leaves.size()) return AMR_ERR_INVALID_ARG;
  long long need = (long long)h->nv * 2 * h->nd * 2 * h->nt;
  if (cap < need) return AMR_ERR_INVALID_ARG;
  CK(h->stagebuf.ensure(std::max<size_t>(h->stagebuf.cap, need * sizeof(double))));
  int rc = with_type(h, [&]<typename real, int ND>() -> int {
    int r = h->ghost_fill_current<real, ND>(h->U0.as<real>());
    if (r) return r;
    cudaError_t e = EulerOps<real, ND>::face_ghosts(h->B, h->U0.as<real>(), h->slabbuf.as<real>(), h->nb.as<int>(),
                                                    (int)leaf, h->stagebuf.as<double>(), h->stream);
    if (e != cudaSuccess) return h->fail_cuda(e, "face_ghosts");
    ++h->launches;
    return AMR_OK;
  });
  if (rc) return rc;
  CK(cudaMemcpyAsync(out, h->stagebuf.p, need * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  return AMR_OK;
}

int amr_march_tuning(amr_handle* h, int* choice, float* us) {
  if (!h || !choice) return AMR_ERR_INVALID_ARG;
  for (int k = 0; k < 3; ++k) {
    choice[2 * k] = h->march_tune[k][0];
    choice[2 * k + 1] = h->march_tune[k][1];
    if (us) us[k] = h->march_us[k];
  }
  return AMR_OK;
}

int amr_set_march_tuning(amr_handle* h, const int* choice) {
  if (!h || !choice) return AMR_ERR_INVALID_ARG;
  for (int k = 0; k < 3; ++k) {
    const int nw = choice[2 * k], p = choice[2 * k + 1];
    if ((nw != 2 && nw != 4 && nw != 8) || (k == 2 && nw != 4) || (p != 0 && p != 1)) return AMR_ERR_INVALID_ARG;
  }
  for (int k = 0; k < 3; ++k) {
    h->march_tune[k][0] = choice[2 * k];
    h->march_tune[k][1] = choice[2 * k + 1];
    h->march_us[k] = 0.f;
  }
  h->march_tuned = true;
  h->drop_graph();
  return AMR_OK;
}

int amr_profile_step(amr_handle* h, double t_end, float* ms, int* kind, int cap, int* nkernels) {
  if (!h || !ms || !kind || !nkernels) return AMR_ERR_INVALID_ARG;
  std::vector<cudaEvent_t> ev;
  std::vector<int> kd;
  cudaEvent_t e0;
  CK(cudaEventCreate(&e0));
  CK(ctl_set_t_end(h->ctl.as<DevCtl>(), t_end, h->stream));
  ++h->launches;
  CK(cudaEventRecord(e0, h->stream));
  h->prof_ev = &ev;
  h->prof_kind = &kd;
  int rc = with_type(h, [&]<typename real, int ND>() -> int { return h->enqueue_step<real, ND>(); });
  h->prof_ev = nullptr;
  h->prof_kind = nullptr;
  cudaError_t es = cudaStreamSynchronize(h->stream);
  int n = (int)kd.size();
  *nkernels = n;
  if (rc == AMR_OK && es == cudaSuccess && n <= cap && ev.size() == 2 * kd.size()) {
    for (int i = 0; i < n; ++i) {
      cudaEventElapsedTime(&ms[i], ev[2 * i], ev[2 * i + 1]);
      kind[i] = kd[i];
    }
  }
  for (auto e : ev) cudaEventDestroy(e);
  cudaEventDestroy(e0);
  if (rc) return rc;
  if (es != cudaSuccess) return h->fail_cuda(es, "profile step");
  if (n > cap) return AMR_ERR_INVALID_ARG;
  return sync_ctl(h);
}

int amr_kernel_launches(const amr_handle* h, long long* n) {
  if (!h || !n) return AMR_ERR_INVALID_ARG;
  *n = h->launches;
  return AMR_OK;
}

}  // extern "C"
