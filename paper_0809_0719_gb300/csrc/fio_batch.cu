// fio_batch.cu -- batches of FIO_F32 plans (fio_batch_* in include/fio.h): the
// step schedule shared by the plans of each (q, s) group, one persistent launch
// per step and group, the two captured CUDA graphs and the launch autotuner.
//
// Schedule of a group (forward): initialization of every member, then p-level
// steps j = 1, 2, ... (member i takes part while j <= lm_i - l0_i, at its level
// l0_i + j), the switch of every member, x-level steps j = 1, 2, ... (while
// j <= l1_i - lm_i, at level lm_i + j) and the termination of every member.  Each
// member keeps its own two state buffers (those of its plan) and alternates
// between them exactly as a single-plan apply does.  The adjoint runs the
// transposed steps in reverse order (Sec. 4 steps conjugate-transposed).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <cstring>
#include <map>
#include <new>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "fio.h"
#include "fio_batch.cuh"
#include "fio_internal.cuh"

namespace fio {
int batch_q3(const BLaunch &, cudaStream_t, int, int *, int *);
int batch_q5(const BLaunch &, cudaStream_t, int, int *, int *);
int batch_q7(const BLaunch &, cudaStream_t, int, int *, int *);
int batch_q9(const BLaunch &, cudaStream_t, int, int *, int *);
int batch_q11(const BLaunch &, cudaStream_t, int, int *, int *);
}  // namespace fio

namespace {

using namespace fio;

int bfail(int code, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return code;
}
int bcuda(int err, const char *what) {
  const cudaError_t e = (cudaError_t)err;
  return bfail(e == cudaErrorMemoryAllocation ? FIO_ENOMEM : FIO_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

int batch_dispatch(const BLaunch &L, cudaStream_t st, int optin, int *blocks_per_sm, int *block) {
  switch (L.q) {
  case 3: return batch_q3(L, st, optin, blocks_per_sm, block);
  case 5: return batch_q5(L, st, optin, blocks_per_sm, block);
  case 7: return batch_q7(L, st, optin, blocks_per_sm, block);
  case 9: return batch_q9(L, st, optin, blocks_per_sm, block);
  case 11: return batch_q11(L, st, optin, blocks_per_sm, block);
  }
  return (int)cudaErrorInvalidValue;
}

__global__ void k_batch_io(BIo *io, const float2 *in, float2 *out) {
  io->in = in;
  io->out = out;
  io->pin = nullptr;
  io->pout = nullptr;
}

// Per-plan user pointers of fio_apply_batch, passed by value in chunks of kPtrChunk plans.
constexpr int kPtrChunk = 1024;
struct PtrChunk {
  const float2 *in[kPtrChunk];
  float2 *out[kPtrChunk];
};
__global__ void k_batch_io_ptrs(BIo *io, const float2 **pin, float2 **pout, int first, int n, PtrChunk c) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    pin[first + i] = c.in[i];
    pout[first + i] = c.out[i];
  }
  if (threadIdx.x == 0) {
    io->in = nullptr;
    io->out = nullptr;
    io->pin = pin;
    io->pout = pout;
  }
}

struct Group {
  int q, s;
  std::vector<int> members;  // plan indices, in batch order
};

// A launch before the device buffer exists: its items live in the host list.
struct HostLaunch {
  BLaunch L;
  size_t item0;  // first item in the host item list
  int blocks_per_sm;
};

long long nb_at(int lb, int e) { return (1LL << lb) << (lb + e); }

}  // namespace

struct fio_batch_s {
  int device = 0, nplans = 0, smem_optin = 0, num_sms = 0;
  std::vector<fio_plan_t> plans;
  std::vector<int> nrhs;
  std::vector<long long> off;
  std::vector<Group> groups;
  std::vector<BWork> items;              // host copy of every launch's items
  std::vector<long long> starts;         // host copy of every launch's start[] arrays
  std::vector<std::vector<HostLaunch>> sched[2];  // [fwd/adj][group] -> launches in order
  void *dev = nullptr;
  BIo *io = nullptr;
  const float2 **pin = nullptr;  // device: per-plan user pointers (fio_apply_batch)
  float2 **pout = nullptr;
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  int parallel = 1, tuned = 0;
  double tune_ms = 0.0;
};

namespace {

// Shared memory of each kernel kind for item set `its` of q, s (dynamic bytes).
long long kind_smem(int kind, int q, int s, int rs, const std::vector<BWork> &its) {
  const long long Q2 = (long long)q * q, M2 = 1LL << (2 * s);
  const long long xd = (long long)sizeof(XDesc);
  long long b = 0;
  switch (kind) {
  case K_INIT:
    for (const BWork &w : its)
      b = std::max(b, ((long long)w.maxsrc * kRMax + (long long)w.GA * w.maxsrc + (long long)w.GA * Q2) * 8 +
                          (long long)w.maxsrc * 2 * q * 4 + (long long)w.GA * ((long long)sizeof(XDesc) + q * 8));
    return b;
  case K_INIT_ADJ:
    for (const BWork &w : its)
      b = std::max(b, ((long long)w.maxsrc * kRMax + w.maxsrc + Q2 + kRMax * Q2) * 8 + (long long)w.maxsrc * 2 * q * 4);
    return b;
  case K_TRANS_P:
  case K_TRANS_X:
  case K_TRANS_P_ADJ:
  case K_TRANS_X_ADJ: return trans32_smem_bytes(q, rs);
  case K_SWITCH:
  case K_SWITCH_ADJ: return sw32_smem_bytes(q);
  case K_TERM: return (2 * kRMax * Q2 + (long long)kRMax * kTermM * q + 2 * (Q2 + kTermM * kTermM)) * 8 + (Q2 + M2) * xd;
  case K_TERM_ADJ:
    return ((long long)kRMax * kTermM * kTermM + (long long)kRMax * q * kTermM + kTermM * kTermM + Q2) * 8 +
           (Q2 + M2) * xd;
  }
  return 0;
}

// Build the forward (adj = 0) or adjoint (adj = 1) schedule of every group.
int build_schedule(fio_batch_s *b, int adj) {
  const int budget = b->smem_optin - (int)sizeof(BWork) - 64;
  b->sched[adj].assign(b->groups.size(), {});
  for (size_t gi = 0; gi < b->groups.size(); gi++) {
    const Group &G = b->groups[gi];
    std::vector<int> cur(b->nplans, 0);
    int maxP = 0, maxX = 0;
    for (int i : G.members) {
      maxP = std::max(maxP, b->plans[i]->d.lm - b->plans[i]->d.l0);
      maxX = std::max(maxX, b->plans[i]->d.l1 - b->plans[i]->d.lm);
    }
    // one step: kind, and for each member whether it takes part and at which level
    auto add = [&](int kind, auto level_of) -> int {
      HostLaunch h;
      memset(&h, 0, sizeof h);
      h.L.kind = kind;
      h.L.q = G.q;
      h.L.s = G.s;
      h.item0 = b->items.size();
      std::vector<BWork> its;
      for (int i : G.members) {
        const int l = level_of(i);
        if (l < 0) continue;
        const PlanDev &d = b->plans[i]->d;
        BWork w;
        memset(&w, 0, sizeof w);
        w.tb = d.tb;
        w.tf = d.tf;
        w.ph = d.ph;
        w.g.L = d.L;
        w.g.e = d.e;
        w.g.q = d.q;
        w.g.s = d.s;
        w.g.l = l;
        w.g.nrhs = b->nrhs[i];
        w.g.rt = kRMax;
        w.g.U = 1;
        w.io_off = b->off[i];
        w.plan = i;
        w.nrt = (b->nrhs[i] + kRMax - 1) / kRMax;
        float2 *S[2] = {(float2 *)d.state[0], (float2 *)d.state[1]};
        switch (kind) {
        case K_INIT:
        case K_INIT_ADJ: {
          w.g.nunits = d.nbox_init;
          w.maxsrc = std::max(1, d.maxsrc);
          int GA = kind == K_INIT ? std::min(kInitChunk, 1 << (2 * d.l0)) : 1;
          std::vector<BWork> one(1, w);
          one[0].GA = GA;
          while (kind == K_INIT && kind_smem(kind, G.q, G.s, 8, one) > budget && GA > 1) one[0].GA = --GA;
          if (kind_smem(kind, G.q, G.s, 8, one) > budget)
            return bfail(FIO_EINVAL, "plan %d: %d sources in one initialization box exceed the batched kernel's shared memory",
                         i, d.maxsrc);
          w.GA = GA;
          if (kind == K_INIT) {
            w.out = S[cur[i]];
          } else {
            w.in = S[cur[i]];
          }
          break;
        }
        case K_SWITCH:
        case K_SWITCH_ADJ:
          w.g.nunits = (1LL << (2 * l)) * nb_at(d.L - l, d.e);
          w.in = S[cur[i]];
          w.out = S[cur[i] ^ 1];
          cur[i] ^= 1;
          break;
        case K_TERM:
          w.g.nunits = 1LL << (2 * l);
          w.in = S[cur[i]];
          break;
        case K_TERM_ADJ:
          w.g.nunits = 1LL << (2 * l);
          w.out = S[cur[i]];
          break;
        default:  // translations
          w.g.nunits = (1LL << (2 * (l - 1))) * nb_at(d.L - l, d.e);
          w.in = S[cur[i]];
          w.out = S[cur[i] ^ 1];
          cur[i] ^= 1;
          break;
        }
        its.push_back(w);
      }
      if (its.empty()) return FIO_OK;
      int maxr = 0;
      for (const BWork &w : its) maxr = std::max(maxr, w.g.nrhs);
      h.L.rs = maxr <= 4 ? 4 : 8;  // translations: narrow subtiles when every plan has few RHS
      const long long sm = kind_smem(kind, G.q, G.s, h.L.rs, its);
      if (sm > budget) return bfail(FIO_EINVAL, "q=%d: the batched kernel needs %lld B of shared memory", G.q, sm);
      h.L.smem = (int)sm;
      h.L.n = (int)its.size();
      h.L.T = b->plans[G.members[0]]->d.T;
      h.L.V = b->plans[G.members[0]]->d.V;
      long long tot = 0;
      for (const BWork &w : its) tot += w.g.nunits * w.nrt;
      h.L.total = tot;
      b->items.insert(b->items.end(), its.begin(), its.end());
      b->sched[adj][gi].push_back(h);
      return FIO_OK;
    };
    int rc;
    const auto &P = b->plans;
    if (!adj) {
      if ((rc = add(K_INIT, [&](int i) { return P[i]->d.l0; }))) return rc;
      for (int j = 1; j <= maxP; j++)
        if ((rc = add(K_TRANS_P, [&](int i) { return j <= P[i]->d.lm - P[i]->d.l0 ? P[i]->d.l0 + j : -1; }))) return rc;
      if ((rc = add(K_SWITCH, [&](int i) { return P[i]->d.lm; }))) return rc;
      for (int j = 1; j <= maxX; j++)
        if ((rc = add(K_TRANS_X, [&](int i) { return j <= P[i]->d.l1 - P[i]->d.lm ? P[i]->d.lm + j : -1; }))) return rc;
      if ((rc = add(K_TERM, [&](int i) { return P[i]->d.l1; }))) return rc;
    } else {
      if ((rc = add(K_TERM_ADJ, [&](int i) { return P[i]->d.l1; }))) return rc;
      for (int j = 1; j <= maxX; j++)
        if ((rc = add(K_TRANS_P_ADJ, [&](int i) { return j <= P[i]->d.l1 - P[i]->d.lm ? P[i]->d.l1 - (j - 1) : -1; })))
          return rc;
      if ((rc = add(K_SWITCH_ADJ, [&](int i) { return P[i]->d.lm; }))) return rc;
      for (int j = 1; j <= maxP; j++)
        if ((rc = add(K_TRANS_X_ADJ, [&](int i) { return j <= P[i]->d.lm - P[i]->d.l0 ? P[i]->d.lm - (j - 1) : -1; })))
          return rc;
      if ((rc = add(K_INIT_ADJ, [&](int i) { return P[i]->d.l0; }))) return rc;
    }
  }
  return FIO_OK;
}

// Capture schedule adj into a graph (groups on parallel branches if parallel).
int build_graph(fio_batch_s *b, int adj, int parallel, cudaGraphExec_t *out) {
  *out = nullptr;
  cudaStream_t cs = nullptr;
  cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return (int)e;
  const size_t ng = b->groups.size();
  const bool fork = parallel && ng > 1;
  std::vector<cudaStream_t> br(fork ? ng : 0, nullptr);
  std::vector<cudaEvent_t> evs(fork ? ng + 1 : 0, nullptr);
  int rc = 0;
  for (auto &s : br)
    if (!rc) rc = (int)cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
  for (auto &v : evs)
    if (!rc) rc = (int)cudaEventCreateWithFlags(&v, cudaEventDisableTiming);
  cudaGraph_t graph = nullptr;
  if (!rc) rc = (int)cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (!rc) {
    int lrc = 0;
    if (fork) {
      cudaEventRecord(evs[ng], cs);
      for (size_t g = 0; g < ng && !lrc; g++) {
        cudaStreamWaitEvent(br[g], evs[ng], 0);
        for (HostLaunch &h : b->sched[adj][g])
          if (!lrc) lrc = batch_dispatch(h.L, br[g], b->smem_optin, nullptr, nullptr);
        cudaEventRecord(evs[g], br[g]);
        cudaStreamWaitEvent(cs, evs[g], 0);
      }
    } else {
      for (size_t g = 0; g < ng && !lrc; g++)
        for (HostLaunch &h : b->sched[adj][g])
          if (!lrc) lrc = batch_dispatch(h.L, cs, b->smem_optin, nullptr, nullptr);
    }
    const cudaError_t ee = cudaStreamEndCapture(cs, &graph);
    rc = lrc ? lrc : (int)ee;
  }
  if (!rc) rc = (int)cudaGraphInstantiate(out, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  for (auto &v : evs)
    if (v) cudaEventDestroy(v);
  for (auto &s : br)
    if (s) cudaStreamDestroy(s);
  cudaStreamDestroy(cs);
  return rc;
}

// Best of `reps` timed runs (after one warm-up) of fn on st, in ms.
template <typename F> float time_ms(cudaStream_t st, F &&fn, int reps = 2) {
  cudaEvent_t a, z;
  cudaEventCreate(&a);
  cudaEventCreate(&z);
  float best = 1e30f;
  for (int rep = 0; rep <= reps; rep++) {
    cudaEventRecord(a, st);
    if (fn()) {
      best = 1e30f;
      break;
    }
    cudaEventRecord(z, st);
    cudaEventSynchronize(z);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, z);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(z);
  return best;
}

void destroy_batch(fio_batch_s *b) {
  if (!b) return;
  cudaDeviceSynchronize();
  for (auto &x : b->exec)
    if (x) cudaGraphExecDestroy(x);
  if (b->dev) cudaFree(b->dev);
  delete b;
}

// Batches built by fio_apply_batch, keyed by the plans' serial numbers and the RHS
// counts; an entry is dropped when one of its plans is destroyed.
struct CachedBatch {
  std::vector<unsigned long long> serials;
  std::vector<int> nrhs;
  fio_batch_s *b;
};
std::mutex g_cache_mu;
std::vector<CachedBatch> g_cache;
constexpr size_t kCacheMax = 8;

}  // namespace

namespace fio {
void batch_cache_forget(fio_plan_t p) {
  std::vector<fio_batch_s *> drop;
  {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    for (size_t i = 0; i < g_cache.size();) {
      bool has = false;
      for (unsigned long long sn : g_cache[i].serials) has = has || sn == p->serial;
      if (has) {
        drop.push_back(g_cache[i].b);
        g_cache.erase(g_cache.begin() + i);
      } else {
        i++;
      }
    }
  }
  for (fio_batch_s *b : drop) destroy_batch(b);
}
}  // namespace fio

extern "C" {

int fio_batch_create(fio_batch_t *out, int nplans, const fio_plan_t *plans, const int *nrhs, int flags) {
  if (!out) return bfail(FIO_EINVAL, "out is NULL");
  *out = nullptr;
  if (nplans < 1 || nplans > 4096) return bfail(FIO_EINVAL, "nplans=%d outside [1, 4096]", nplans);
  if (!plans || !nrhs) return bfail(FIO_EINVAL, "NULL plans or nrhs");
  if (flags & ~(FIO_BATCH_TUNE | FIO_BATCH_SERIAL)) return bfail(FIO_EINVAL, "unknown flags 0x%x", flags);
  int dev = -1;
  cudaError_t ce = cudaGetDevice(&dev);
  if (ce != cudaSuccess) return bfail(FIO_EDEVICE, "no CUDA device: %s", cudaGetErrorString(ce));
  std::set<fio_plan_t> seen;
  for (int i = 0; i < nplans; i++) {
    const fio_plan_t p = plans[i];
    if (!p) return bfail(FIO_EINVAL, "plan %d is NULL", i);
    if (!seen.insert(p).second) return bfail(FIO_EINVAL, "plan %d appears twice", i);
    if (p->device != dev) return bfail(FIO_EINVAL, "plan %d was built on device %d, device %d is current", i, p->device, dev);
    if (p->d.precision != FIO_F32 || !p->d.tf.xnode) return bfail(FIO_EINVAL, "plan %d is not an FIO_F32 plan", i);
    if (nrhs[i] < 1 || nrhs[i] > p->d.nrhs_max)
      return bfail(FIO_EINVAL, "nrhs[%d]=%d outside [1, %d]", i, nrhs[i], p->d.nrhs_max);
    if ((1 << p->d.s) > kTermM) return bfail(FIO_EINVAL, "plan %d: 2^s=%d exceeds %d", i, 1 << p->d.s, kTermM);
  }
  fio_batch_s *b = new (std::nothrow) fio_batch_s();
  if (!b) return bfail(FIO_ENOMEM, "host allocation failed");
  b->device = dev;
  b->nplans = nplans;
  b->parallel = (flags & FIO_BATCH_SERIAL) ? 0 : 1;
  b->plans.assign(plans, plans + nplans);
  b->nrhs.assign(nrhs, nrhs + nplans);
  cudaDeviceGetAttribute(&b->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
  b->off.assign(nplans + 1, 0);
  for (int i = 0; i < nplans; i++) b->off[i + 1] = b->off[i] + (long long)nrhs[i] * b->plans[i]->d.N * b->plans[i]->d.N;
  std::map<std::pair<int, int>, int> gid;
  for (int i = 0; i < nplans; i++) {
    const auto key = std::make_pair(b->plans[i]->d.q, b->plans[i]->d.s);
    auto it = gid.find(key);
    if (it == gid.end()) {
      it = gid.emplace(key, (int)b->groups.size()).first;
      b->groups.push_back(Group{key.first, key.second, {}});
    }
    b->groups[it->second].members.push_back(i);
  }
  int rc;
  for (int adj = 0; adj < 2; adj++)
    if ((rc = build_schedule(b, adj))) {
      destroy_batch(b);
      return rc;
    }
  // one device buffer: io slot | items | start arrays | per-plan in and out pointers
  size_t nstart = 0;
  for (int adj = 0; adj < 2; adj++)
    for (auto &gl : b->sched[adj])
      for (HostLaunch &h : gl) nstart += h.L.n + 1;
  const size_t o_items = 256, o_start = (o_items + b->items.size() * sizeof(BWork) + 255) & ~(size_t)255;
  const size_t o_ptrs = (o_start + nstart * sizeof(long long) + 255) & ~(size_t)255;
  const size_t bytes = o_ptrs + 2 * (size_t)b->nplans * sizeof(void *);
  if ((ce = cudaMalloc(&b->dev, bytes)) != cudaSuccess) {
    destroy_batch(b);
    return bcuda((int)ce, "cudaMalloc(batch descriptors)");
  }
  b->io = (BIo *)b->dev;
  b->pin = (const float2 **)((char *)b->dev + o_ptrs);
  b->pout = (float2 **)(b->pin + b->nplans);
  BWork *d_items = (BWork *)((char *)b->dev + o_items);
  long long *d_start = (long long *)((char *)b->dev + o_start);
  size_t si = 0;
  for (int adj = 0; adj < 2; adj++)
    for (auto &gl : b->sched[adj])
      for (HostLaunch &h : gl) {
        h.L.items = d_items + h.item0;
        h.L.start = d_start + si;
        h.L.io = b->io;
        long long acc = 0;
        for (int k = 0; k < h.L.n; k++) {
          b->starts.push_back(acc);
          const BWork &w = b->items[h.item0 + k];
          acc += w.g.nunits * w.nrt;
        }
        b->starts.push_back(acc);
        si += h.L.n + 1;
      }
  const BIo io0 = {nullptr, nullptr};
  ce = cudaMemcpy(b->dev, &io0, sizeof io0, cudaMemcpyHostToDevice);
  if (ce == cudaSuccess)
    ce = cudaMemcpy(d_items, b->items.data(), b->items.size() * sizeof(BWork), cudaMemcpyHostToDevice);
  if (ce == cudaSuccess) ce = cudaMemcpy(d_start, b->starts.data(), b->starts.size() * sizeof(long long), cudaMemcpyHostToDevice);
  if (ce != cudaSuccess) {
    destroy_batch(b);
    return bcuda((int)ce, "cudaMemcpy(batch descriptors)");
  }
  // default grids: every resident CTA slot once (persistent), at most the work
  for (int adj = 0; adj < 2; adj++)
    for (auto &gl : b->sched[adj])
      for (HostLaunch &h : gl) {
        int bps = 0, blk = 0;
        if ((rc = batch_dispatch(h.L, nullptr, b->smem_optin, &bps, &blk))) {
          destroy_batch(b);
          return bcuda(rc, "batched kernel occupancy");
        }
        if (bps < 1) {
          destroy_batch(b);
          return bfail(FIO_EINVAL, "a batched kernel (q=%d) cannot be resident with %d B of shared memory", h.L.q, h.L.smem);
        }
        h.blocks_per_sm = bps;
        h.L.grid = (int)std::min<long long>(h.L.total, (long long)bps * b->num_sms);
      }
  if (flags & FIO_BATCH_TUNE) {
    const auto t0 = std::chrono::steady_clock::now();
    b->tuned = 1;
    void *scratch = nullptr;
    const size_t sb = (size_t)b->off[nplans] * 8 + 256;
    if ((ce = cudaMalloc(&scratch, 2 * sb)) != cudaSuccess) {
      destroy_batch(b);
      return bcuda((int)ce, "cudaMalloc(tuning scratch)");
    }
    cudaMemset(scratch, 0, 2 * sb);
    cudaStream_t ts = nullptr;
    cudaStreamCreateWithFlags(&ts, cudaStreamNonBlocking);
    k_batch_io<<<1, 1, 0, ts>>>(b->io, (const float2 *)scratch, (float2 *)((char *)scratch + sb));
    for (int adj = 0; adj < 2; adj++)
      for (auto &gl : b->sched[adj])
        for (HostLaunch &h : gl) {
          const bool is_trans = h.L.kind == K_TRANS_P || h.L.kind == K_TRANS_X || h.L.kind == K_TRANS_P_ADJ ||
                                h.L.kind == K_TRANS_X_ADJ;
          BLaunch best_l = h.L;
          float best = 1e30f;
          for (int rs : {4, 8}) {
            if (!is_trans && rs != h.L.rs) continue;
            BLaunch L = h.L;
            L.rs = rs;
            if (is_trans) {
              std::vector<BWork> none;
              L.smem = (int)kind_smem(L.kind, L.q, L.s, rs, none);
            }
            int bps = 0, blk = 0;
            if (batch_dispatch(L, nullptr, b->smem_optin, &bps, &blk) || bps < 1) continue;
            const long long g1 = (long long)bps * b->num_sms;
            std::vector<long long> cand = {g1, 2 * g1, 4 * g1};
            if (L.total <= 8 * g1) cand.push_back(L.total);  // one CTA per unit
            for (long long c : cand) {
              L.grid = (int)std::min<long long>(c, L.total);
              const float ms = time_ms(ts, [&]() { return batch_dispatch(L, ts, b->smem_optin, nullptr, nullptr); });
              if (ms < best) {
                best = ms;
                best_l = L;
              }
            }
          }
          h.L = best_l;
        }
    // groups on parallel branches or one after another
    if (b->groups.size() > 1 && b->parallel) {
      float t[2] = {1e30f, 1e30f};
      for (int par = 0; par < 2; par++) {
        cudaGraphExec_t ex = nullptr;
        if (build_graph(b, 0, par, &ex) == 0) {
          t[par] = time_ms(ts, [&]() { return (int)cudaGraphLaunch(ex, ts); });
          cudaStreamSynchronize(ts);
          cudaGraphExecDestroy(ex);
        }
      }
      b->parallel = t[1] <= t[0] ? 1 : 0;
    }
    cudaStreamSynchronize(ts);
    ce = cudaGetLastError();
    cudaStreamDestroy(ts);
    cudaFree(scratch);
    b->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    if (ce != cudaSuccess) {
      destroy_batch(b);
      return bcuda((int)ce, "batch autotuning");
    }
  }
  for (int adj = 0; adj < 2; adj++)
    if ((rc = build_graph(b, adj, b->parallel, &b->exec[adj]))) {
      destroy_batch(b);
      return bcuda(rc, "batch graph capture");
    }
  *out = b;
  set_last_error("");
  return FIO_OK;
}

int fio_batch_destroy(fio_batch_t b) {
  destroy_batch(b);
  return FIO_OK;
}

int fio_batch_offsets(fio_batch_t b, long long *off) {
  if (!b || !off) return bfail(FIO_EINVAL, "NULL argument");
  for (int i = 0; i <= b->nplans; i++) off[i] = b->off[i];
  return FIO_OK;
}

static int batch_io(fio_batch_t b, const void *in, void *out, cudaStream_t st) {
  if (!b) return bfail(FIO_EINVAL, "batch is NULL");
  if (!in || !out) return bfail(FIO_EINVAL, "NULL data pointer");
  if (((uintptr_t)in | (uintptr_t)out) & 15) return bfail(FIO_EINVAL, "data pointers must be 16-byte aligned");
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != b->device) return bfail(FIO_EINVAL, "batch was built on device %d but device %d is current", b->device, dev);
  k_batch_io<<<1, 1, 0, st>>>(b->io, (const float2 *)in, (float2 *)out);
  const cudaError_t ce = cudaGetLastError();
  return ce == cudaSuccess ? FIO_OK : bcuda((int)ce, "batch io kernel");
}

int fio_batch_apply(fio_batch_t b, const void *in, void *out, int adjoint, void *stream) {
  cudaStream_t st = (cudaStream_t)stream;
  int rc = batch_io(b, in, out, st);
  if (rc) return rc;
  const cudaError_t ce = cudaGraphLaunch(b->exec[adjoint ? 1 : 0], st);
  return ce == cudaSuccess ? FIO_OK : bcuda((int)ce, "cudaGraphLaunch");
}

static int apply_batch_ptrs(fio_plan_t *plans, int nplans, const void *const *in, void *const *out,
                            const int *nrhs, int adjoint, void *stream) {
  if (!plans || !in || !out || !nrhs) return bfail(FIO_EINVAL, "NULL plans, data pointer arrays or nrhs");
  if (nplans < 1 || nplans > 4096) return bfail(FIO_EINVAL, "nplans=%d outside [1, 4096]", nplans);
  for (int i = 0; i < nplans; i++) {
    if (!plans[i]) return bfail(FIO_EINVAL, "plan %d is NULL", i);
    if (!in[i] || !out[i]) return bfail(FIO_EINVAL, "data pointer %d is NULL", i);
    if (((uintptr_t)in[i] | (uintptr_t)out[i]) & 15) return bfail(FIO_EINVAL, "data pointers %d are not 16-byte aligned", i);
  }
  cudaStream_t st = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lk(g_cache_mu);
  fio_batch_s *b = nullptr;
  for (CachedBatch &c : g_cache) {
    if ((int)c.serials.size() != nplans) continue;
    bool same = true;
    for (int i = 0; i < nplans && same; i++) same = c.serials[i] == plans[i]->serial && c.nrhs[i] == nrhs[i];
    if (same) b = c.b;
  }
  if (!b) {
    int rc = fio_batch_create(&b, nplans, plans, nrhs, 0);
    if (rc) return rc;
    if (g_cache.size() >= kCacheMax) {
      destroy_batch(g_cache.front().b);
      g_cache.erase(g_cache.begin());
    }
    CachedBatch c;
    for (int i = 0; i < nplans; i++) c.serials.push_back(plans[i]->serial);
    c.nrhs.assign(nrhs, nrhs + nplans);
    c.b = b;
    g_cache.push_back(c);
  }
  int dev = -1;
  cudaGetDevice(&dev);
  if (dev != b->device) return bfail(FIO_EINVAL, "plans were built on device %d but device %d is current", b->device, dev);
  for (int first = 0; first < nplans; first += kPtrChunk) {
    const int n = std::min(kPtrChunk, nplans - first);
    PtrChunk c;
    for (int i = 0; i < n; i++) {
      c.in[i] = (const float2 *)in[first + i];
      c.out[i] = (float2 *)out[first + i];
    }
    k_batch_io_ptrs<<<1, 256, 0, st>>>(b->io, b->pin, b->pout, first, n, c);
  }
  cudaError_t ce = cudaGetLastError();
  if (ce != cudaSuccess) return bcuda((int)ce, "batch pointer kernel");
  ce = cudaGraphLaunch(b->exec[adjoint ? 1 : 0], st);
  return ce == cudaSuccess ? FIO_OK : bcuda((int)ce, "cudaGraphLaunch");
}

int fio_apply_batch(fio_plan_t *plans, int nplans, const void *const *f, void *const *u, const int *nrhs,
                    void *stream) {
  return apply_batch_ptrs(plans, nplans, f, u, nrhs, 0, stream);
}

int fio_apply_batch_adjoint(fio_plan_t *plans, int nplans, const void *const *g, void *const *fbar, const int *nrhs,
                            void *stream) {
  return apply_batch_ptrs(plans, nplans, g, fbar, nrhs, 1, stream);
}

int fio_batch_info(fio_batch_t b, fio_batch_info_t *info) {
  if (!b || !info) return bfail(FIO_EINVAL, "NULL argument");
  memset(info, 0, sizeof *info);
  info->nplans = b->nplans;
  info->ngroups = (int)b->groups.size();
  for (int adj = 0; adj < 2; adj++) {
    int n = 0;
    for (auto &gl : b->sched[adj]) n += (int)gl.size();
    (adj ? info->launches_adj : info->launches_fwd) = n;
  }
  info->parallel_groups = b->parallel;
  info->tuned = b->tuned;
  info->total_elems = b->off[b->nplans];
  info->tune_ms = b->tune_ms;
  return FIO_OK;
}

int fio_batch_profile(fio_batch_t b, const void *in, void *out, int adjoint, void *stream, fio_kernel_time_t *times,
                      int max, int *n) {
  if (!times || !n) return bfail(FIO_EINVAL, "NULL argument");
  *n = 0;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = batch_io(b, in, out, st);
  if (rc) return rc;
  const int adj = adjoint ? 1 : 0;
  size_t nl = 0;
  for (auto &gl : b->sched[adj]) nl += gl.size();
  std::vector<cudaEvent_t> ev(2 * nl, nullptr);
  for (auto &v : ev)
    if (cudaEventCreate(&v) != cudaSuccess) return bcuda((int)cudaGetLastError(), "cudaEventCreate");
  std::vector<int> kinds;
  size_t k = 0;
  for (auto &gl : b->sched[adj])
    for (HostLaunch &h : gl) {
      cudaEventRecord(ev[2 * k], st);
      if ((rc = batch_dispatch(h.L, st, b->smem_optin, nullptr, nullptr))) break;
      cudaEventRecord(ev[2 * k + 1], st);
      kinds.push_back(h.L.kind);
      k++;
    }
  cudaError_t ce = cudaStreamSynchronize(st);
  double ms[kKinds] = {0};
  long long cnt[kKinds] = {0};
  for (size_t i = 0; i < k && ce == cudaSuccess && !rc; i++) {
    float t = 0.f;
    cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
    ms[kinds[i]] += t;
    cnt[kinds[i]]++;
  }
  for (auto &v : ev) cudaEventDestroy(v);
  if (rc) return bcuda(rc, "batched launch");
  if (ce != cudaSuccess) return bcuda((int)ce, "cudaStreamSynchronize");
  for (int kk = 0; kk < kKinds && *n < max; kk++) {
    if (!cnt[kk]) continue;
    fio_kernel_time_t &o = times[(*n)++];
    snprintf(o.name, sizeof o.name, "b_%s", kKernelNames[kk]);
    o.launches = cnt[kk];
    o.ms = ms[kk];
  }
  return FIO_OK;
}

}  // extern "C"
