// Batched form: many independent two-field (SH, F) split-step simulations of
// uneven grids, mismatch and crystal length, run from one CUDA graph launch
// in one of two forms, which the autotuner chooses between by timing both:
//
// Grouped.  The instances of one grid shape are stored one after another, so
// that a pass of all of them is one launch of the single-instance kernels
// (the y- and tau-passes see the instances' fields as more fields; the x-pass
// takes each instance's step, coupling and mismatch from a table).  Per shape
// the instances are ordered by step count, longest first, so the ones still
// running at step j are a prefix: step j is four launches over that prefix.
// Each shape's launch sequence runs on a stream of its own inside the graph,
// so the passes of different shapes overlap (a DRAM-bound pass of one beside
// an issue-bound pass of another).  Any shape the single-instance path
// supports (ny, nt >= 2) can join.
//
// Persistent (the four compiled shapes below only): ONE persistent
// cooperative kernel advances every instance.
//
// Work queue.  Each instance's propagation is a fixed sequence of passes:
//   x(first half step of step 0), then per step j: y-forward, tau-propagator,
//   y-inverse, x(second half of j + first half of j+1, or the last half).
// Each pass is cut into CTA-sized items.  An instance's items are numbered in
// that order; a CTA takes the next item of an instance with one atomicAdd on
// the instance's counter.  An item of pass q may start only when every item
// of pass q-1 of the same instance has completed (per-instance pass barrier:
// one completion counter per pass, release/acquire at GPU scope).  Items only
// wait on items with smaller numbers, which are held by running CTAs, and all
// CTAs are co-resident (cooperative launch), so the scheduler cannot
// deadlock.  Every wait is bounded by a %globaltimer limit: on expiry the
// kernel records BRAHMS_E_TIMEOUT and exits.  CTAs scan instances in
// longest-first order (grid points x steps), so the longest chains start first
// and small instances fill the gaps.
//
// Shapes (NX = NY, NT) are compiled in: (32,64), (64,128), (96,192), (128,256).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "alloc_hook.h"
#include "brahms.h"
#include "kernels.cuh"

namespace brahms {
namespace {

constexpr int kBT = 256;  // threads per persistent CTA
constexpr int kTypeX = 0, kTypeYF = 1, kTypeT = 2, kTypeYI = 3;

struct Shape {
  int nxy, nt;
};
constexpr Shape kShapes[] = {{32, 64}, {64, 128}, {96, 192}, {128, 256}};
constexpr int kNumShapes = 4;

template <int S>
struct ShapeT {
  static constexpr int NXY = kShapes[S].nxy;
  static constexpr int NT = kShapes[S].nt;
  using PY = FftPlan<NXY>;
  using PT = TauPlan<NT>;
  static constexpr int YTPC = tiles_per_cta_t<PY, kBT>();
  static constexpr int TTPC = tiles_per_cta_t<PT, kBT>();
  static constexpr int smem_floats2() {
    const int x = xtile_smem_floats2<NXY, kBT>(2);
    const int y = 2 * tw_table_size<PY>() + YTPC * NXY * ColTile<PY>::value;
    const int t = 2 * tw_table_size<PT>() + TTPC * NT * ColTile<PT>::value;
    return x > y ? (x > t ? x : t) : (y > t ? y : t);
  }
};

constexpr int batch_smem_floats2() {
  int m = 0;
  m = ShapeT<0>::smem_floats2() > m ? ShapeT<0>::smem_floats2() : m;
  m = ShapeT<1>::smem_floats2() > m ? ShapeT<1>::smem_floats2() : m;
  m = ShapeT<2>::smem_floats2() > m ? ShapeT<2>::smem_floats2() : m;
  m = ShapeT<3>::smem_floats2() > m ? ShapeT<3>::smem_floats2() : m;
  return m;
}

struct InstDev {
  float2* state;
  const float2* ecoef;  // stage factors of every x-pass: [step + 1][6] (see stage_table)
  long long fstride;
  const float4 *twx, *twt;  // NX = NY: one table serves x and y
  const float2 *px, *py, *pt;
  int nx, ny, nt, shape;
  int nz;
  double dz, dk;
  float kh[2], kh2[2];
  float scale, scale_lo;
  int n_x, n_y, n_t;      // items per pass type
  int g_x, g_y, g_t;      // CTA tiles per item (tile granularity)
  long long ct_x, ct_y, ct_t;  // CTA tiles per pass type
  long long total;        // items in the whole propagation
  long long done_off;     // first completion counter of this instance
};

struct BatchArgs {
  const InstDev* inst;  // longest first
  int ninst;
  unsigned long long* next;  // per instance item counter
  unsigned int* done;        // per instance, per pass completion counters
  int* status;               // 0 ok, BRAHMS_E_TIMEOUT
  unsigned long long timeout_ns;
};

__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_relaxed64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct Item {
  int type;   // kTypeX ...
  int step;   // z-step j the pass belongs to (x: the step whose second half it applies, -1 for the first pass)
  long long q;  // pass number
  long long tile;  // first CTA tile
  long long ntiles;  // CTA tiles in this item
};

__device__ __forceinline__ long long pass_items(const InstDev& I, long long q) {
  if (q == 0) return I.n_x;
  const int sub = (int)((q - 1) % 4);
  return sub == 0 || sub == 2 ? I.n_y : (sub == 1 ? I.n_t : I.n_x);
}

__device__ __forceinline__ Item decode(const InstDev& I, long long k) {
  Item it;
  long long r;
  if (k < I.n_x) {
    it.type = kTypeX;
    it.step = -1;
    it.q = 0;
    r = k;
  } else {
    const long long G = 2LL * I.n_y + I.n_t + I.n_x;
    const long long k2 = k - I.n_x;
    const long long j = k2 / G;
    r = k2 % G;
    it.step = (int)j;
    int sub;
    if (r < I.n_y) {
      sub = 0;
    } else if (r < (long long)I.n_y + I.n_t) {
      sub = 1;
      r -= I.n_y;
    } else if (r < 2LL * I.n_y + I.n_t) {
      sub = 2;
      r -= I.n_y + I.n_t;
    } else {
      sub = 3;
      r -= 2LL * I.n_y + I.n_t;
    }
    it.type = sub == 0 ? kTypeYF : (sub == 1 ? kTypeT : (sub == 2 ? kTypeYI : kTypeX));
    it.q = 1 + 4 * j + sub;
  }
  const int g = it.type == kTypeX ? I.g_x : (it.type == kTypeT ? I.g_t : I.g_y);
  const long long ct = it.type == kTypeX ? I.ct_x : (it.type == kTypeT ? I.ct_t : I.ct_y);
  it.tile = r * g;
  it.ntiles = (it.tile + g <= ct) ? g : ct - it.tile;
  return it;
}

// ---------------------------------------------------------------- items
template <int S>
__device__ __noinline__ void run_item(const InstDev& I, const Item& it, float4* sm4) {
  using SH = ShapeT<S>;
  constexpr int NXY = SH::NXY, NT = SH::NT;
  float4* tw = sm4;
  if (it.type == kTypeX) {
    XPassArgs p{};
    p.data = I.state;
    p.fstride = I.fstride;
    p.rows = (long long)NXY * NT;
    p.tw = I.twx;
    p.dz = I.dz;
    for (int f = 0; f < 2; ++f) {
      p.kh[f] = I.kh[f];
      p.kh2[f] = I.kh2[f];
    }
    p.scale = 1.f;
    if (it.step < 0) {
      p.mode = XM_NL_FIRST;
      p.phiA = 0.0;
      p.dkA = I.dk;
    } else {
      p.mode = it.step < I.nz - 1 ? XM_NL_MID : XM_NL_LAST;
      p.phiB = I.dk * (it.step * I.dz);
      p.dkB = I.dk;
      p.phiA = I.dk * ((it.step + 1) * I.dz);
      p.dkA = I.dk;
    }
    float2* coef = reinterpret_cast<float2*>(sm4);
    float2* rowbuf = coef + 12;
    if (threadIdx.x < 6) coef[threadIdx.x] = I.ecoef[(it.step + 1) * 6 + threadIdx.x];
    __syncthreads();
    for (long long c = 0; c < it.ntiles; ++c) {
      xpass_tile<NXY, 2, kBT>(p, it.tile + c, coef, rowbuf);
      __syncthreads();
    }
    return;
  }
  AxisArgs a{};
  a.data = I.state;
  a.nx = NXY;
  a.ny = NXY;
  a.nt = NT;
  a.fstride = I.fstride;
  a.px = I.px;
  a.py = I.py;
  a.pt = I.pt;
  a.scale = I.scale;
  a.scale_lo = I.scale_lo;
  if (it.type == kTypeT) {
    a.xtiles = (NXY + ColTile<typename SH::PT>::value - 1) / ColTile<typename SH::PT>::value;
    a.ntiles = 2LL * NXY * a.xtiles;
    a.tw = I.twt;
    float2* xch = reinterpret_cast<float2*>(tw + tw_table_size<typename SH::PT>());
    for (int i = threadIdx.x; i < tw_table_size<typename SH::PT>(); i += kBT) tw[i] = I.twt[i];
    __syncthreads();
    for (long long c = 0; c < it.ntiles; ++c) {
      tprop_tile<typename SH::PT, kBT>(a, it.tile + c, TwShared{tw}, xch);
      __syncthreads();
    }
  } else {
    a.xtiles = (NXY + ColTile<typename SH::PY>::value - 1) / ColTile<typename SH::PY>::value;
    a.ntiles = 2LL * NT * a.xtiles;
    a.tw = I.twx;
    float2* xch = reinterpret_cast<float2*>(tw + tw_table_size<typename SH::PY>());
    for (int i = threadIdx.x; i < tw_table_size<typename SH::PY>(); i += kBT) tw[i] = I.twx[i];
    __syncthreads();
    for (long long c = 0; c < it.ntiles; ++c) {
      if (it.type == kTypeYF) axis_tile<typename SH::PY, false, 1, kBT>(a, it.tile + c, TwShared{tw}, xch);
      else axis_tile<typename SH::PY, true, 1, kBT>(a, it.tile + c, TwShared{tw}, xch);
      __syncthreads();
    }
  }
}

// Warp 0: find and claim the next runnable item.  The lanes look at 32
// instances at a time (one L2 round trip per 32 instead of per instance);
// the runnable candidate of lowest index -- the longest-first order -- takes
// one atomicAdd on its counter, and on a lost race the next candidate is
// tried.  The lane that wins writes the item to shared memory.  Returns, to
// every lane, 1 with an item, 0 when no instance has items left, -1 on
// timeout.
__device__ int claim_warp(const BatchArgs& b, unsigned long long t_start, int* s_inst, Item* s_item) {
  const int lane = threadIdx.x & 31;
  for (;;) {
    bool any_left = false;
    for (int base = 0; base < b.ninst; base += 32) {
      const int i = base + lane;
      bool cand = false, left = false;
      if (i < b.ninst) {
        const InstDev& I = b.inst[i];
        const unsigned long long w = ld_relaxed64(b.next + i);
        if ((long long)w < I.total) {
          left = true;
          const Item peek = decode(I, (long long)w);
          cand = peek.q == 0 || ld_acquire(b.done + I.done_off + peek.q - 1) >= pass_items(I, peek.q - 1);
        }
      }
      any_left = __any_sync(0xffffffffu, left) || any_left;
      unsigned m = __ballot_sync(0xffffffffu, cand);
      while (m) {
        const int src = __ffs(m) - 1;
        int got = 0;
        if (lane == src) {
          const InstDev& I = b.inst[i];
          const unsigned long long k = atomicAdd(b.next + i, 1ULL);
          if ((long long)k < I.total) {
            const Item it = decode(I, (long long)k);
            got = 1;
            if (it.q > 0) {
              // the item may belong to the next pass when others claimed concurrently
              while (ld_acquire(b.done + I.done_off + it.q - 1) < pass_items(I, it.q - 1)) {
                if (gtimer() - t_start > b.timeout_ns) {
                  got = -1;
                  break;
                }
                __nanosleep(64);
              }
            }
            *s_inst = i;
            *s_item = it;
          }
        }
        got = __shfl_sync(0xffffffffu, got, src);
        if (got != 0) return got;
        m &= m - 1;
      }
    }
    if (!any_left) return 0;
    if (gtimer() - t_start > b.timeout_ns) return -1;
    __nanosleep(128);
  }
}

// Warp 0 claims the next item while warp 1 publishes the completion of the
// previous one (fence + release), so the two round trips overlap.
__global__ void __launch_bounds__(kBT, 2) batch_kernel(const BatchArgs b) {
  extern __shared__ float4 sm4[];
  __shared__ int s_inst, s_state;
  __shared__ Item s_item;
  long long prev = -1;  // completion counter of the previous item (thread 32)
  for (;;) {
    if (threadIdx.x < 32) {
      // the timeout covers one claim: the time a CTA may wait for runnable work
      const int r = claim_warp(b, gtimer(), &s_inst, &s_item);
      __syncwarp();
      if (threadIdx.x == 0) {
        if (r < 0) atomicExch(b.status, (int)BRAHMS_E_TIMEOUT);
        if (r > 0 && ld_acquire(reinterpret_cast<const unsigned int*>(b.status)) != 0) s_state = 0;
        else s_state = r;
      }
    } else if (threadIdx.x == 32 && prev >= 0) {
      __threadfence();
      red_release_add(b.done + prev, 1u);
    }
    __syncthreads();
    if (s_state <= 0) break;
    const InstDev& I = b.inst[s_inst];
    const Item it = s_item;
    switch (I.shape) {
      case 0: run_item<0>(I, it, sm4); break;
      case 1: run_item<1>(I, it, sm4); break;
      case 2: run_item<2>(I, it, sm4); break;
      default: run_item<3>(I, it, sm4); break;
    }
    __syncthreads();  // the item's stores are issued; s_item may be rewritten
    prev = I.done_off + it.q;
  }
}

int shape_of(int nx, int ny, int nt) {
  for (int s = 0; s < kNumShapes; ++s)
    if (kShapes[s].nxy == nx && kShapes[s].nxy == ny && kShapes[s].nt == nt) return s;
  return -1;
}
int xtile_rows_of(int s) {
  switch (s) {
    case 0: return xtile_rows<32, kBT>();
    case 1: return xtile_rows<64, kBT>();
    case 2: return xtile_rows<96, kBT>();
    default: return xtile_rows<128, kBT>();
  }
}
int ytpc_of(int s) {
  switch (s) {
    case 0: return ShapeT<0>::YTPC;
    case 1: return ShapeT<1>::YTPC;
    case 2: return ShapeT<2>::YTPC;
    default: return ShapeT<3>::YTPC;
  }
}
int ttpc_of(int s) {
  switch (s) {
    case 0: return ShapeT<0>::TTPC;
    case 1: return ShapeT<1>::TTPC;
    case 2: return ShapeT<2>::TTPC;
    default: return ShapeT<3>::TTPC;
  }
}

constexpr double kTwoPi = 6.283185307179586476925286766559;

}  // namespace
}  // namespace brahms

using namespace brahms;

struct BatchInstHost {
  int nx, ny, nt, shape, nz;  // shape: index into the persistent kernel's shapes, -1 if not one of them
  double dx, dy, dt, dz, dk, d_eff;
  brahms_field_params fp[2];
  char* mem = nullptr;  // state + tables until the instance joins a group (then NULL)
  float2* state = nullptr;
  float4 *twx = nullptr, *twt = nullptr;
  float2 *px = nullptr, *py = nullptr, *pt = nullptr;
  const float2* ecoef = nullptr;  // its stage factors in its group's table, [step + 1][6]
  bool have_fields = false;
  long long npoints() const { return (long long)nx * ny * nt; }
};

// The instances of one grid shape, stored one after another in sorted order
// (step count, longest first): state [slot][2][nt][ny][nx], propagator
// tables [2 slot + f][n] per axis, the shape's twiddles, the per-instance
// table of the grouped x-pass.
struct BatchGroup {
  int nx, ny, nt;
  std::vector<int> members;  // instance indices in slot order
  char* mem = nullptr;
  float2* state = nullptr;
  float2 *px = nullptr, *py = nullptr, *pt = nullptr;
  float4 *twx = nullptr, *twy = nullptr, *twt = nullptr;
  GroupInst* params = nullptr;
  float2* ecoef = nullptr;  // stage factors [slot][steps + 1][6]
  int ecoef_steps = 0;      // steps per slot in the table (the group's largest nz)
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  long long npoints() const { return (long long)nx * ny * nt; }
};

enum { kModeAuto = 0, kModeGrouped = 1, kModePersistent = 2 };

struct brahms_batch {
  cudaStream_t stream = nullptr;
  std::vector<BatchInstHost> inst;
  std::vector<BatchGroup> groups;
  bool layout_dirty = true;
  int mode = kModeAuto;   // asked for (brahms_batch_set_mode)
  int chosen = kModeGrouped;  // what an automatic mode runs (set by the tuner)
  cudaEvent_t ev_fork = nullptr;
  std::string err;
  int gran[kNumShapes][3];  // tiles per item (x, y, t) per shape
  int ctas_per_sm = 1;
  // device scheduling state
  InstDev* d_inst = nullptr;
  unsigned long long* d_next = nullptr;
  unsigned int* d_done = nullptr;
  int* d_status = nullptr;
  int* h_status = nullptr;  // pinned
  size_t done_count = 0;
  std::vector<int> order;  // longest first
  // graph
  cudaGraphExec_t exec = nullptr;
  bool dirty = true;
  int nz_cap = 0;  // > 0: every instance runs min(nz, nz_cap) steps (autotuning runs)
  int grid = 0;
  size_t smem = 0;
  double timeout_s = 5.0;
  long long launches = 0;        // kernel launches made by graph launches so far
  long long graph_launches = 0;  // kernel launches in one graph launch
};

namespace {

brahms_status bfail(brahms_batch* b, brahms_status s, const std::string& m) {
  if (b) b->err = m;
  return s;
}
#define BB_CK(call)                                                                                  \
  do {                                                                                               \
    cudaError_t e_ = (call);                                                                         \
    if (e_ != cudaSuccess) return bfail(b, BRAHMS_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// an allocation that failed is BRAHMS_E_OOM (the batch stays usable)
#define BB_ALLOC(call)                                                      \
  do {                                                                      \
    if ((call) != cudaSuccess) {                                            \
      cudaGetLastError();                                                   \
      return bfail(b, BRAHMS_E_OOM, std::string(#call) + ": out of memory"); \
    }                                                                       \
  } while (0)

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

void free_device(brahms_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  b->exec = nullptr;
  cudaFree(b->d_inst);
  cudaFree(b->d_next);
  cudaFree(b->d_done);
  b->d_inst = nullptr;
  b->d_next = nullptr;
  b->d_done = nullptr;
  b->d_status = nullptr;  // lives in d_done's allocation
}

void free_groups(brahms_batch* b) {
  for (auto& g : b->groups) {
    cudaFree(g.mem);
    if (g.stream) cudaStreamDestroy(g.stream);
    if (g.done) cudaEventDestroy(g.done);
  }
  b->groups.clear();
}

brahms_status build_tables_for(brahms_batch* b, BatchInstHost& I);

bool persistent_possible(const brahms_batch* b) {
  for (auto& I : b->inst)
    if (I.shape < 0) return false;
  return true;
}

int effective_nz(const brahms_batch* b, const BatchInstHost& I) {
  return b->nz_cap > 0 ? std::min(I.nz, b->nz_cap) : I.nz;
}

// The stage factors e^{+i Phi} of every x-pass of every instance of a group,
// [slot][step + 1][6] (step -1: the first half step), formed on the host in
// FP64 exactly as the single-instance path forms them: the same phase
// accumulation Phi_{j+1} = Phi_j + dk dz and the same reduction
// (fill_stage_factors), so a batched instance computes what
// brahms_propagate computes, bit for bit.
cudaError_t stage_table(brahms_batch* b, BatchGroup& g) {
  const int S = g.ecoef_steps + 1;
  std::vector<float2> h((size_t)6 * S * g.members.size(), make_float2(1.f, 0.f));
  for (size_t slot = 0; slot < g.members.size(); ++slot) {
    const BatchInstHost& I = b->inst[g.members[slot]];
    XPassArgs x{};
    x.dz = I.dz;
    double phi = 0.0;
    for (int j = -1; j < I.nz; ++j) {
      if (j < 0) {
        x.phiB = x.dkB = 0.0;
        x.phiA = phi;
        x.dkA = I.dk;
      } else {
        x.phiB = phi;
        x.dkB = I.dk;
        phi += I.dk * I.dz;
        x.phiA = phi;
        x.dkA = I.dk;
      }
      fill_stage_factors(x);
      for (int s = 0; s < 6; ++s) h[((size_t)slot * S + (j + 1)) * 6 + s] = x.ecoef[s];
    }
  }
  cudaError_t e = cudaMemcpyAsync(g.ecoef, h.data(), sizeof(float2) * h.size(), cudaMemcpyHostToDevice, b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);  // h is a local buffer
  return e;
}

// Group the instances by shape into arrays of their own (see BatchGroup):
// the fields move there, the tables are rebuilt there, and every instance's
// pointers (used by both forms) point into its group.
brahms_status layout(brahms_batch* b) {
  std::vector<BatchGroup> gs;
  for (int i = 0; i < (int)b->inst.size(); ++i) {
    const BatchInstHost& I = b->inst[i];
    int g = -1;
    for (int k = 0; k < (int)gs.size(); ++k)
      if (gs[k].nx == I.nx && gs[k].ny == I.ny && gs[k].nt == I.nt) g = k;
    if (g < 0) {
      gs.push_back(BatchGroup{});
      g = (int)gs.size() - 1;
      gs[g].nx = I.nx;
      gs[g].ny = I.ny;
      gs[g].nt = I.nt;
    }
    gs[g].members.push_back(i);
  }
  auto release = [&](brahms_status s) {
    for (auto& g : gs) {
      cudaFree(g.mem);
      if (g.stream) cudaStreamDestroy(g.stream);
      if (g.done) cudaEventDestroy(g.done);
    }
    return s;
  };
  for (auto& g : gs) {
    std::stable_sort(g.members.begin(), g.members.end(),
                     [&](int a, int c) { return b->inst[a].nz > b->inst[c].nz; });
    const size_t m = g.members.size(), n = (size_t)g.npoints();
    size_t off = 0;
    auto take = [&](size_t bytes) {
      size_t o = off;
      off += al256(bytes);
      return o;
    };
    const size_t o_state = take(sizeof(float2) * 2 * n * m), o_px = take(sizeof(float2) * 2 * m * g.nx),
                 o_py = take(sizeof(float2) * 2 * m * g.ny), o_pt = take(sizeof(float2) * 2 * m * g.nt),
                 o_twx = take(sizeof(float4) * tw_table_size_of(g.nx)),
                 o_twy = take(sizeof(float4) * tw_table_size_of(g.ny)),
                 o_twt = take(sizeof(float4) * tw_table_size_of(g.nt)), o_par = take(sizeof(GroupInst) * m);
    g.ecoef_steps = 0;
    for (int i : g.members) g.ecoef_steps = std::max(g.ecoef_steps, b->inst[i].nz);
    const size_t o_coef = take(sizeof(float2) * 6 * (size_t)(g.ecoef_steps + 1) * m);
    if (dev_alloc((void**)&g.mem, off) != cudaSuccess) {
      cudaGetLastError();
      return release(bfail(b, BRAHMS_E_OOM, "batch group memory"));
    }
    g.state = (float2*)(g.mem + o_state);
    g.px = (float2*)(g.mem + o_px);
    g.py = (float2*)(g.mem + o_py);
    g.pt = (float2*)(g.mem + o_pt);
    g.twx = (float4*)(g.mem + o_twx);
    g.twy = (float4*)(g.mem + o_twy);
    g.twt = (float4*)(g.mem + o_twt);
    g.params = (GroupInst*)(g.mem + o_par);
    g.ecoef = (float2*)(g.mem + o_coef);
    if (cudaStreamCreateWithFlags(&g.stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming) != cudaSuccess)
      return release(bfail(b, BRAHMS_E_CUDA, "group stream"));
    cudaError_t e = upload_twiddles(g.twx, g.nx, b->stream);
    if (e == cudaSuccess) e = upload_twiddles(g.twy, g.ny, b->stream);
    if (e == cudaSuccess) e = upload_twiddles(g.twt, g.nt, b->stream);
    if (e == cudaSuccess) e = stage_table(b, g);
    if (e != cudaSuccess) return release(bfail(b, BRAHMS_E_CUDA, std::string("twiddles: ") + cudaGetErrorString(e)));
    for (size_t slot = 0; slot < m; ++slot) {
      BatchInstHost& I = b->inst[g.members[slot]];
      float2* dst = g.state + slot * 2 * n;
      if (I.have_fields && I.state) {
        e = cudaMemcpyAsync(dst, I.state, sizeof(float2) * 2 * n, cudaMemcpyDeviceToDevice, b->stream);
        if (e != cudaSuccess) return release(bfail(b, BRAHMS_E_CUDA, cudaGetErrorString(e)));
      }
    }
  }
  // the copies out of the old locations are done before those are released
  if (cudaStreamSynchronize(b->stream) != cudaSuccess) return release(bfail(b, BRAHMS_E_CUDA, "layout copy"));
  free_groups(b);
  for (auto& g : gs) {
    const size_t n = (size_t)g.npoints();
    for (size_t slot = 0; slot < g.members.size(); ++slot) {
      BatchInstHost& I = b->inst[g.members[slot]];
      if (I.mem) cudaFree(I.mem);
      I.mem = nullptr;
      I.state = g.state + slot * 2 * n;
      I.px = g.px + slot * 2 * g.nx;
      I.py = g.py + slot * 2 * g.ny;
      I.pt = g.pt + slot * 2 * g.nt;
      I.twx = g.twx;
      I.twt = g.twt;
      I.ecoef = g.ecoef + slot * (size_t)(g.ecoef_steps + 1) * 6;
      brahms_status st = build_tables_for(b, I);
      if (st != BRAHMS_OK) {
        b->groups = gs;
        return st;
      }
    }
  }
  b->groups = gs;
  b->layout_dirty = false;
  return BRAHMS_OK;
}

// one graph launch: per group, on the group's stream, the first x-pass of
// every instance, then per step j the y-forward, tau-propagator, y-inverse
// and x-pass of the instances still running at step j
brahms_status prepare_grouped(brahms_batch* b) {
  BB_CK(cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming)) ;
  for (auto& g : b->groups) {
    std::vector<GroupInst> h(g.members.size());
    for (size_t slot = 0; slot < g.members.size(); ++slot) {
      const BatchInstHost& I = b->inst[g.members[slot]];
      GroupInst& p = h[slot];
      for (int f = 0; f < 2; ++f) {
        double k = kTwoPi * I.d_eff / (I.fp[f].n * I.fp[f].lambda);
        if (f == 0) k *= 0.5;  // degenerate SHG: 1/2 on the SH equation
        p.kh[f] = (float)(k * 0.5 * I.dz);
        p.kh2[f] = 0.5f * p.kh[f];
      }
      p.dk = I.dk;
      p.dz = I.dz;
      p.nz = effective_nz(b, I);
    }
    BB_CK(cudaMemcpyAsync(g.params, h.data(), sizeof(GroupInst) * h.size(), cudaMemcpyHostToDevice, b->stream));
    BB_CK(cudaStreamSynchronize(b->stream));  // h is a local buffer
  }
  // configure every kernel outside the capture (no work: empty ranges)
  for (auto& g : b->groups) {
    AxisArgs z{};
    z.nx = g.nx;
    z.ny = g.ny;
    z.nt = g.nt;
    z.xtiles = 1;
    BB_CK(run_axis_fft(g.ny, 1, false, z, b->stream));
    BB_CK(run_axis_fft(g.ny, 1, true, z, b->stream));
    BB_CK(run_tpass_prop(g.nt, z, b->stream));
    XPassArgs x{};
    BB_CK(run_xpass_group(g.nx, x, g.params, g.ecoef, 6, 0, 0, b->stream));
    BB_CK(run_xpass(g.nx, 2, x, b->stream));
  }
  cudaStream_t cap = nullptr;
  BB_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaEventRecord(b->ev_fork, cap);
  long long nl = 0;
  for (auto& g : b->groups) {
    if (e != cudaSuccess) break;
    cudaStream_t s = g.stream;
    e = cudaStreamWaitEvent(s, b->ev_fork, 0);
    const long long n = g.npoints();
    const int m = (int)g.members.size();
    const int rows = xpass_rows_of(g.nx);
    const bool whole = rows > 0 && ((long long)g.ny * g.nt) % rows == 0;
    std::vector<int> nzs(m);
    int nz_max = 0;
    for (int slot = 0; slot < m; ++slot) {
      nzs[slot] = effective_nz(b, b->inst[g.members[slot]]);
      nz_max = std::max(nz_max, nzs[slot]);
    }
    XPassArgs base{};
    base.data = g.state;
    base.fstride = n;
    base.rows = (long long)g.ny * g.nt;
    base.tw = g.twx;
    base.scale = 1.f;
    base.ny = g.ny;
    // an x-pass over the first a slots (per instance where an instance's rows
    // do not fill whole CTAs)
    auto xpass = [&](int step, int a) -> cudaError_t {
      if (whole) return run_xpass_group(g.nx, base, g.params, g.ecoef, (g.ecoef_steps + 1) * 6, step, a, s);
      for (int slot = 0; slot < a; ++slot) {
        const BatchInstHost& I = b->inst[g.members[slot]];
        XPassArgs p = base;
        p.data = g.state + (long long)slot * 2 * n;
        p.dz = I.dz;
        for (int f = 0; f < 2; ++f) {
          double k = kTwoPi * I.d_eff / (I.fp[f].n * I.fp[f].lambda);
          if (f == 0) k *= 0.5;
          p.kh[f] = (float)(k * 0.5 * I.dz);
          p.kh2[f] = 0.5f * p.kh[f];
        }
        // the phase accumulated as brahms_propagate accumulates it
        double phi = 0.0;
        for (int j = 0; j < step; ++j) phi += I.dk * I.dz;
        if (step < 0) {
          p.mode = XM_NL_FIRST;
          p.phiA = 0.0;
          p.dkA = I.dk;
        } else {
          p.mode = step == nzs[slot] - 1 ? XM_NL_LAST : XM_NL_MID;
          p.phiB = phi;
          p.dkB = I.dk;
          p.phiA = phi + I.dk * I.dz;
          p.dkA = I.dk;
        }
        cudaError_t ee = run_xpass(g.nx, 2, p, s);
        if (ee != cudaSuccess) return ee;
      }
      return cudaSuccess;
    };
    AxisArgs ay{};
    ay.data = g.state;
    ay.nx = g.nx;
    ay.ny = g.ny;
    ay.nt = g.nt;
    ay.fstride = n;
    ay.xtiles = (g.nx + col_tile_of(g.ny) - 1) / col_tile_of(g.ny);
    ay.tw = g.twy;
    AxisArgs at = ay;
    at.xtiles = (g.nx + tau_col_tile_of(g.nt) - 1) / tau_col_tile_of(g.nt);
    at.tw = g.twt;
    at.px = g.px;
    at.py = g.py;
    at.pt = g.pt;
    const double inv_n = 1.0 / (double)n;
    at.scale = (float)inv_n;
    at.scale_lo = (float)(inv_n - (double)at.scale);
    if (e == cudaSuccess) e = xpass(-1, m);
    nl += whole ? 1 : m;
    int a = m;
    for (int j = 0; j < nz_max && e == cudaSuccess; ++j) {
      while (a > 0 && nzs[a - 1] <= j) --a;  // slots still running at step j
      ay.ntiles = 2LL * a * g.nt * ay.xtiles;
      at.ntiles = 2LL * a * g.ny * at.xtiles;
      e = run_axis_fft(g.ny, 1, false, ay, s);
      if (e == cudaSuccess) e = run_tpass_prop(g.nt, at, s);
      if (e == cudaSuccess) e = run_axis_fft(g.ny, 1, true, ay, s);
      if (e == cudaSuccess) e = xpass(j, a);
      nl += 3 + (whole ? 1 : a);
    }
    if (e == cudaSuccess) e = cudaEventRecord(g.done, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cap, g.done, 0);
  }
  cudaError_t e2 = cudaStreamEndCapture(cap, &graph);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) return bfail(b, BRAHMS_E_CUDA, std::string("grouped graph: ") + cudaGetErrorString(e));
  b->graph_launches = nl;
  b->grid = 0;
  b->dirty = false;
  return BRAHMS_OK;
}

int run_mode(const brahms_batch* b) { return b->mode == kModeAuto ? b->chosen : b->mode; }

brahms_status prepare_persistent(brahms_batch* b);

brahms_status prepare(brahms_batch* b) {
  if (!b->dirty) return BRAHMS_OK;
  free_device(b);
  if (b->ev_fork) {
    cudaEventDestroy(b->ev_fork);
    b->ev_fork = nullptr;
  }
  if (b->inst.empty()) return bfail(b, BRAHMS_E_STATE, "empty batch");
  for (auto& I : b->inst)
    if (!I.have_fields) return bfail(b, BRAHMS_E_STATE, "an instance has no fields");
  if (b->layout_dirty) {
    brahms_status s = layout(b);
    if (s != BRAHMS_OK) return s;
  }
  if (run_mode(b) == kModeGrouped || !persistent_possible(b)) return prepare_grouped(b);
  return prepare_persistent(b);
}

brahms_status prepare_persistent(brahms_batch* b) {
  const int n = (int)b->inst.size();
  if (n == 0) return bfail(b, BRAHMS_E_STATE, "empty batch");
  for (auto& I : b->inst)
    if (!I.have_fields) return bfail(b, BRAHMS_E_STATE, "an instance has no fields");
  // longest first: grid points x steps
  b->order.resize(n);
  for (int i = 0; i < n; ++i) b->order[i] = i;
  std::stable_sort(b->order.begin(), b->order.end(), [&](int a, int c) {
    return b->inst[a].npoints() * b->inst[a].nz > b->inst[c].npoints() * b->inst[c].nz;
  });
  std::vector<InstDev> h(n);
  long long off = 0;
  for (int r = 0; r < n; ++r) {
    const BatchInstHost& I = b->inst[b->order[r]];
    InstDev& d = h[r];
    d.state = I.state;
    d.ecoef = I.ecoef;
    d.fstride = I.npoints();
    d.twx = I.twx;
    d.twt = I.twt;
    d.px = I.px;
    d.py = I.py;
    d.pt = I.pt;
    d.nx = I.nx;
    d.ny = I.ny;
    d.nt = I.nt;
    d.shape = I.shape;
    d.nz = b->nz_cap > 0 ? std::min(I.nz, b->nz_cap) : I.nz;
    d.dz = I.dz;
    d.dk = I.dk;
    for (int f = 0; f < 2; ++f) {
      double k = kTwoPi * I.d_eff / (I.fp[f].n * I.fp[f].lambda);
      if (f == 0) k *= 0.5;
      d.kh[f] = (float)(k * 0.5 * I.dz);
      d.kh2[f] = 0.5f * d.kh[f];
    }
    const double inv_n = 1.0 / (double)I.npoints();
    d.scale = (float)inv_n;
    d.scale_lo = (float)(inv_n - (double)d.scale);
    const int rows = xtile_rows_of(I.shape);
    d.ct_x = ((long long)I.ny * I.nt + rows - 1) / rows;
    const long long ytiles = 2LL * I.nt * ((I.nx + col_tile_of(I.ny) - 1) / col_tile_of(I.ny));
    const long long ttiles = 2LL * I.ny * ((I.nx + tau_col_tile_of(I.nt) - 1) / tau_col_tile_of(I.nt));
    d.ct_y = (ytiles + ytpc_of(I.shape) - 1) / ytpc_of(I.shape);
    d.ct_t = (ttiles + ttpc_of(I.shape) - 1) / ttpc_of(I.shape);
    d.g_x = b->gran[I.shape][0];
    d.g_y = b->gran[I.shape][1];
    d.g_t = b->gran[I.shape][2];
    d.n_x = (int)((d.ct_x + d.g_x - 1) / d.g_x);
    d.n_y = (int)((d.ct_y + d.g_y - 1) / d.g_y);
    d.n_t = (int)((d.ct_t + d.g_t - 1) / d.g_t);
    d.total = (long long)d.n_x + (long long)d.nz * (2LL * d.n_y + d.n_t + d.n_x);
    d.done_off = off;
    off += 1 + 4LL * d.nz;
  }
  b->done_count = (size_t)off;
  BB_ALLOC(dev_alloc((void**)&b->d_inst, sizeof(InstDev) * n));
  BB_ALLOC(dev_alloc((void**)&b->d_next, sizeof(unsigned long long) * n));
  BB_ALLOC(dev_alloc((void**)&b->d_done, al256(sizeof(unsigned int) * b->done_count) + 256));
  b->d_status = reinterpret_cast<int*>(reinterpret_cast<char*>(b->d_done) + al256(sizeof(unsigned int) * b->done_count));
  BB_CK(cudaMemcpy(b->d_inst, h.data(), sizeof(InstDev) * n, cudaMemcpyHostToDevice));
  // launch shape: all CTAs co-resident
  b->smem = (size_t)batch_smem_floats2() * sizeof(float2);
  BB_CK(cudaFuncSetAttribute(batch_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
  int per_sm = 0, sms = 0, dev = 0;
  BB_CK(cudaGetDevice(&dev));
  BB_CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BB_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel, kBT, b->smem));
  if (per_sm < 1) return bfail(b, BRAHMS_E_CUDA, "batched kernel cannot be resident");
  b->grid = sms * std::min(per_sm, b->ctas_per_sm);
  // capture: reset counters, run the persistent kernel
  BatchArgs args{};
  args.inst = b->d_inst;
  args.ninst = n;
  args.next = b->d_next;
  args.done = b->d_done;
  args.status = b->d_status;
  args.timeout_ns = (unsigned long long)(b->timeout_s * 1e9);
  cudaStream_t cap = nullptr;
  BB_CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_next, 0, sizeof(unsigned long long) * n, cap);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_done, 0, al256(sizeof(unsigned int) * b->done_count) + sizeof(int), cap);
  if (e == cudaSuccess) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = dim3(b->grid);
    cfg.blockDim = dim3(kBT);
    cfg.dynamicSmemBytes = b->smem;
    cfg.stream = cap;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, batch_kernel, args);
  }
  cudaError_t e2 = cudaStreamEndCapture(cap, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess) return bfail(b, BRAHMS_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  b->graph_launches = 1;
  b->dirty = false;
  return BRAHMS_OK;
}

brahms_status build_tables_for(brahms_batch* b, BatchInstHost& I) {
  TableArgs a{};
  a.px = I.px;
  a.py = I.py;
  a.pt = I.pt;
  a.nx = I.nx;
  a.ny = I.ny;
  a.nt = I.nt;
  a.nf = 2;
  a.dx = I.dx;
  a.dy = I.dy;
  a.dt = I.dt;
  a.dz = I.dz;
  for (int f = 0; f < 2; ++f) {
    a.k[f] = kTwoPi * I.fp[f].n / I.fp[f].lambda;
    a.rho[f] = I.fp[f].rho;
    a.delta[f] = I.fp[f].delta;
    a.k2[f] = I.fp[f].k2;
    a.k3[f] = I.fp[f].k3;
    a.alpha[f] = I.fp[f].alpha;
  }
  BB_CK(run_prop_tables(a, b->stream));
  BB_CK(upload_twiddles(I.twx, I.nx, b->stream));
  BB_CK(upload_twiddles(I.twt, I.nt, b->stream));
  b->launches += 1;
  return BRAHMS_OK;
}

}  // namespace

extern "C" {

brahms_status brahms_batch_create(brahms_batch** out, void* cuda_stream) {
  if (!out) return BRAHMS_E_ARG;
  brahms_batch* b = new brahms_batch();
  b->stream = (cudaStream_t)cuda_stream;
  for (int s = 0; s < kNumShapes; ++s)
    for (int k = 0; k < 3; ++k) b->gran[s][k] = 1;
  if (pinned_alloc((void**)&b->h_status, sizeof(int)) != cudaSuccess) {
    delete b;
    return BRAHMS_E_OOM;
  }
  *out = b;
  return BRAHMS_OK;
}

void brahms_batch_free(brahms_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  free_device(b);
  free_groups(b);
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  for (auto& I : b->inst) cudaFree(I.mem);
  cudaFreeHost(b->h_status);
  delete b;
}

const char* brahms_batch_last_error(const brahms_batch* b) { return b ? b->err.c_str() : "no batch"; }

brahms_status brahms_batch_add(brahms_batch* b, int nx, int ny, int nt, double dx, double dy, double dt,
                               const brahms_field_params* fp, double d_eff, double dk, int nz, double dz,
                               int* index) {
  if (!b) return BRAHMS_E_ARG;
  if (!fp) return bfail(b, BRAHMS_E_ARG, "fp is NULL");
  if (!size_supported(nx) || !size_supported(ny) || !size_supported(nt) || ny < 2 || nt < 2)
    return bfail(b, BRAHMS_E_SIZE, "batched grid lengths: the FFT lengths of the single-instance path, ny, nt >= 2");
  if (b->mode == kModePersistent && shape_of(nx, ny, nt) < 0)
    return bfail(b, BRAHMS_E_SIZE, "the persistent form runs the shapes (nx=ny, nt) in {(32,64),(64,128),(96,192),(128,256)} only");
  const int s = shape_of(nx, ny, nt);
  if (!(dx > 0) || !(dy > 0) || !(dt > 0) || !(dz > 0) || nz < 1 || !std::isfinite(dk) || !std::isfinite(d_eff) ||
      !std::isfinite(dz))
    return bfail(b, BRAHMS_E_ARG, "bad spacing, step or mismatch");
  BatchInstHost I;
  I.nx = nx;
  I.ny = ny;
  I.nt = nt;
  I.shape = s;
  I.nz = nz;
  I.dx = dx;
  I.dy = dy;
  I.dt = dt;
  I.dz = dz;
  I.dk = dk;
  I.d_eff = d_eff;
  I.fp[0] = fp[0];
  I.fp[1] = fp[1];
  const size_t n = (size_t)I.npoints();
  size_t o_state = 0, o_twx = al256(sizeof(float2) * 2 * n),
         o_twt = o_twx + al256(sizeof(float4) * tw_table_size_of(nx)),
         o_px = o_twt + al256(sizeof(float4) * tw_table_size_of(nt)), o_py = o_px + al256(sizeof(float2) * 2 * nx),
         o_pt = o_py + al256(sizeof(float2) * 2 * ny), total = o_pt + al256(sizeof(float2) * 2 * nt);
  if (dev_alloc((void**)&I.mem, total) != cudaSuccess) {
    cudaGetLastError();
    return bfail(b, BRAHMS_E_OOM, "device allocation failed");
  }
  I.state = (float2*)(I.mem + o_state);
  I.twx = (float4*)(I.mem + o_twx);
  I.twt = (float4*)(I.mem + o_twt);
  I.px = (float2*)(I.mem + o_px);
  I.py = (float2*)(I.mem + o_py);
  I.pt = (float2*)(I.mem + o_pt);
  brahms_status st = build_tables_for(b, I);
  if (st != BRAHMS_OK) {
    cudaFree(I.mem);
    return st;
  }
  b->inst.push_back(I);
  b->dirty = true;
  b->layout_dirty = true;
  if (index) *index = (int)b->inst.size() - 1;
  return BRAHMS_OK;
}

brahms_status brahms_batch_set_fields(brahms_batch* b, int index, const void* const* fields, int dtype,
                                      int on_device) {
  if (!b) return BRAHMS_E_ARG;
  if (index < 0 || index >= (int)b->inst.size()) return bfail(b, BRAHMS_E_ARG, "bad instance index");
  if (!fields || !fields[0] || !fields[1]) return bfail(b, BRAHMS_E_ARG, "fields is NULL");
  if (dtype != BRAHMS_C64) return bfail(b, BRAHMS_E_ARG, "batched fields must be complex64");
  BatchInstHost& I = b->inst[index];
  const size_t n = (size_t)I.npoints();
  for (int f = 0; f < 2; ++f)
    BB_CK(cudaMemcpyAsync(I.state + f * n, fields[f], sizeof(float2) * n,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, b->stream));
  if (!on_device) BB_CK(cudaStreamSynchronize(b->stream));
  if (!I.have_fields) b->dirty = true;
  I.have_fields = true;
  return BRAHMS_OK;
}

brahms_status brahms_batch_set_granularity(brahms_batch* b, int shape, int gx, int gy, int gt) {
  if (!b) return BRAHMS_E_ARG;
  if (shape < 0 || shape >= kNumShapes || gx < 1 || gy < 1 || gt < 1 || gx > 64 || gy > 64 || gt > 64)
    return bfail(b, BRAHMS_E_ARG, "bad granularity");
  b->gran[shape][0] = gx;
  b->gran[shape][1] = gy;
  b->gran[shape][2] = gt;
  b->dirty = true;
  return BRAHMS_OK;
}

brahms_status brahms_batch_set_timeout(brahms_batch* b, double seconds) {
  if (!b) return BRAHMS_E_ARG;
  if (!(seconds >= 0.0) || !(seconds <= 3600.0)) return bfail(b, BRAHMS_E_ARG, "timeout must be in [0, 3600] s");
  b->timeout_s = seconds;
  b->dirty = true;  // the limit is an argument of the captured launch
  return BRAHMS_OK;
}

brahms_status brahms_batch_run(brahms_batch* b) {
  if (!b) return BRAHMS_E_ARG;
  brahms_status s = prepare(b);
  if (s != BRAHMS_OK) return s;
  BB_CK(cudaGraphLaunch(b->exec, b->stream));
  b->launches += b->graph_launches;
  return BRAHMS_OK;
}

brahms_status brahms_batch_set_mode(brahms_batch* b, int mode) {
  if (!b) return BRAHMS_E_ARG;
  if (mode != kModeAuto && mode != kModeGrouped && mode != kModePersistent)
    return bfail(b, BRAHMS_E_ARG, "mode: 0 automatic, 1 grouped, 2 persistent");
  if (mode == kModePersistent && !persistent_possible(b))
    return bfail(b, BRAHMS_E_SIZE, "the persistent form runs the shapes (nx=ny, nt) in {(32,64),(64,128),(96,192),(128,256)} only");
  b->mode = mode;
  b->dirty = true;
  return BRAHMS_OK;
}

int brahms_batch_get_mode(const brahms_batch* b) {
  if (!b) return -1;
  const int m = b->mode == kModeAuto ? b->chosen : b->mode;
  return (m == kModePersistent && !persistent_possible(b)) ? kModeGrouped : m;
}

brahms_status brahms_batch_sync(brahms_batch* b) {
  if (!b) return BRAHMS_E_ARG;
  BB_CK(cudaStreamSynchronize(b->stream));
  if (b->d_status) {
    BB_CK(cudaMemcpy(b->h_status, b->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (*b->h_status != 0) return bfail(b, BRAHMS_E_TIMEOUT, "persistent kernel gave up waiting for a pass");
  }
  return BRAHMS_OK;
}

brahms_status brahms_batch_get_fields(brahms_batch* b, int index, void* const* out, int dtype, int on_device) {
  if (!b) return BRAHMS_E_ARG;
  if (index < 0 || index >= (int)b->inst.size()) return bfail(b, BRAHMS_E_ARG, "bad instance index");
  if (!out || !out[0] || !out[1]) return bfail(b, BRAHMS_E_ARG, "out is NULL");
  if (dtype != BRAHMS_C64) return bfail(b, BRAHMS_E_ARG, "batched fields are complex64");
  BatchInstHost& I = b->inst[index];
  const size_t n = (size_t)I.npoints();
  for (int f = 0; f < 2; ++f)
    BB_CK(cudaMemcpyAsync(out[f], I.state + f * n, sizeof(float2) * n,
                          on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, b->stream));
  return brahms_batch_sync(b);
}

brahms_status brahms_batch_info(const brahms_batch* b, int* ninstances, int* grid, int* threads,
                                long long* launches) {
  if (!b) return BRAHMS_E_ARG;
  if (ninstances) *ninstances = (int)b->inst.size();
  if (grid) *grid = b->grid;
  if (threads) *threads = kBT;
  if (launches) *launches = b->launches;
  return BRAHMS_OK;
}

// Autotuner: the whole batch is timed with every instance capped at
// tune_steps steps, the fields saved before and restored after every trial.
// The grouped form is timed once; the persistent form (when its shapes allow
// it) is searched: for each shape the tiles per item, then the CTAs per SM.
// With the automatic mode the faster of the two forms is kept.
brahms_status brahms_batch_tune(brahms_batch* b, int tune_steps, double* best_ms) {
  if (!b) return BRAHMS_E_ARG;
  if (b->inst.empty()) return bfail(b, BRAHMS_E_STATE, "empty batch");
  for (auto& I : b->inst)
    if (!I.have_fields) return bfail(b, BRAHMS_E_STATE, "an instance has no fields");
  if (tune_steps < 1) tune_steps = 16;
  size_t bytes = 0;
  for (auto& I : b->inst) bytes += sizeof(float2) * 2 * (size_t)I.npoints();
  char* save = nullptr;
  BB_ALLOC(dev_alloc((void**)&save, bytes));
  auto copy_all = [&](bool to_save) -> cudaError_t {
    size_t o = 0;
    for (auto& I : b->inst) {
      const size_t n = sizeof(float2) * 2 * (size_t)I.npoints();
      cudaError_t e = to_save ? cudaMemcpyAsync(save + o, I.state, n, cudaMemcpyDeviceToDevice, b->stream)
                              : cudaMemcpyAsync(I.state, save + o, n, cudaMemcpyDeviceToDevice, b->stream);
      if (e != cudaSuccess) return e;
      o += n;
    }
    return cudaSuccess;
  };
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  auto trial = [&](float* ms) -> brahms_status {
    b->dirty = true;
    brahms_status s = prepare(b);
    if (s != BRAHMS_OK) return s;
    float best = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      BB_CK(copy_all(false));
      BB_CK(cudaEventRecord(e0, b->stream));
      BB_CK(cudaGraphLaunch(b->exec, b->stream));
      BB_CK(cudaEventRecord(e1, b->stream));
      s = brahms_batch_sync(b);
      if (s != BRAHMS_OK) return s;
      float t = 0.f;
      BB_CK(cudaEventElapsedTime(&t, e0, e1));
      best = std::min(best, t);
    }
    *ms = best;
    return BRAHMS_OK;
  };
  brahms_status st = BRAHMS_OK;
  cudaError_t ce = copy_all(true);
  if (ce != cudaSuccess) st = bfail(b, BRAHMS_E_CUDA, cudaGetErrorString(ce));
  b->nz_cap = tune_steps;
  const bool try_grouped = b->mode != kModePersistent;
  const bool try_persistent = b->mode != kModeGrouped && persistent_possible(b);
  float grouped_ms = 1e30f;
  const int chosen0 = b->chosen;
  if (try_grouped && st == BRAHMS_OK) {
    b->chosen = kModeGrouped;
    st = trial(&grouped_ms);
  }
  if (try_persistent) b->chosen = kModePersistent;
  bool present[kNumShapes] = {};
  for (auto& I : b->inst)
    if (I.shape >= 0) present[I.shape] = true;
  float cur = 0.f;
  if (try_persistent && st == BRAHMS_OK) st = trial(&cur);
  for (int sh = 0; sh < kNumShapes && st == BRAHMS_OK && try_persistent; ++sh) {
    if (!present[sh]) continue;
    int keep[3] = {b->gran[sh][0], b->gran[sh][1], b->gran[sh][2]};
    // one granularity for all three passes, then a per-pass search
    for (int g : {1, 2, 4, 8, 16}) {
      if (g == keep[0] && g == keep[1] && g == keep[2]) continue;
      b->gran[sh][0] = b->gran[sh][1] = b->gran[sh][2] = g;
      float ms = 0.f;
      st = trial(&ms);
      if (st != BRAHMS_OK) break;
      if (ms < cur) {
        cur = ms;
        keep[0] = keep[1] = keep[2] = g;
      }
    }
    // per pass: keep doubling (then halving) while the batch gets faster
    for (int k = 0; k < 3 && st == BRAHMS_OK; ++k) {
      for (int up = 1; up >= 0 && st == BRAHMS_OK; --up) {
        for (;;) {
          const int g = up ? keep[k] * 2 : keep[k] / 2;
          if (g < 1 || g > 64) break;
          for (int j = 0; j < 3; ++j) b->gran[sh][j] = keep[j];
          b->gran[sh][k] = g;
          float ms = 0.f;
          st = trial(&ms);
          if (st != BRAHMS_OK || ms >= cur) break;
          cur = ms;
          keep[k] = g;
        }
      }
    }
    b->gran[sh][0] = keep[0];
    b->gran[sh][1] = keep[1];
    b->gran[sh][2] = keep[2];
  }
  if (st == BRAHMS_OK && try_persistent) {
    const int keep = b->ctas_per_sm;
    for (int c : {1, 2}) {
      if (c == keep) continue;
      b->ctas_per_sm = c;
      float ms = 0.f;
      st = trial(&ms);
      if (st != BRAHMS_OK) break;
      if (ms < cur) cur = ms;
      else b->ctas_per_sm = keep;
    }
  }
  if (st == BRAHMS_OK) {
    if (!try_persistent) {
      b->chosen = kModeGrouped;
      cur = grouped_ms;
    } else if (try_grouped && grouped_ms <= cur) {
      b->chosen = kModeGrouped;
      cur = grouped_ms;
    }
  } else {
    b->chosen = chosen0;
  }
  b->nz_cap = 0;
  b->dirty = true;
  cudaError_t re = copy_all(false);
  cudaStreamSynchronize(b->stream);
  cudaFree(save);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st == BRAHMS_OK && re != cudaSuccess) st = bfail(b, BRAHMS_E_CUDA, cudaGetErrorString(re));
  if (best_ms) *best_ms = cur;
  return st;
}

brahms_status brahms_batch_get_schedule(const brahms_batch* b, int shape, int* gx, int* gy, int* gt,
                                        int* ctas_per_sm) {
  if (!b || shape < 0 || shape >= kNumShapes) return BRAHMS_E_ARG;
  if (gx) *gx = b->gran[shape][0];
  if (gy) *gy = b->gran[shape][1];
  if (gt) *gt = b->gran[shape][2];
  if (ctas_per_sm) *ctas_per_sm = b->ctas_per_sm;
  return BRAHMS_OK;
}

}  // extern "C"
