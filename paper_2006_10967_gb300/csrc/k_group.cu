// Stepping a group of fields with one launch per kernel per RK stage
// (C ABI: fr_group_create, fr_group_step, fr_group_destroy).
//
// The ensemble of uneven instances is one batch field per order (one union
// mesh per order, per-element time steps and parameters).  A group launch
// covers all of them: block b of the launch finds its field from the
// cumulative block counts (the work list: field g owns blocks
// [cum[g], cum[g+1])) and runs that order's residual or update body on its
// own tile.  One launch of kb_group and one of ka_group per RK stage, the
// sequence captured in CUDA graphs of kGroupSteps steps; the orders' blocks
// share the GPU in one wave instead of four launches on four streams.
//
// Built for the quad mixed-precision physical step with orders p = 2..5
// (the ensemble's); preconditioning stays per field.
#include <algorithm>
#include <cstring>
#include <new>

#include "field.cuh"
#include "k_tensor_inst.cuh"

namespace frp {

constexpr int kGroupMax = 4;   // orders 2, 3, 4, 5 -> slots 0..3
constexpr int kGroupPmin = 2;

struct GroupArgs {
  int cum[kGroupMax + 1];      // cumulative block counts per slot
  KArgs a[kGroupMax];          // the slot's field arguments (unused when empty)
};

template <typename LYF>
struct GMax {
  static constexpr int t3 = LYF::template L<3>::THREADS, t4 = LYF::template L<4>::THREADS,
                       t5 = LYF::template L<5>::THREADS, t6 = LYF::template L<6>::THREADS;
  static constexpr int THREADS = std::max(std::max(t3, t4), std::max(t5, t6));
  static constexpr size_t SMEM = std::max(std::max(LYF::template L<3>::SMEM, LYF::template L<4>::SMEM),
                                          std::max(LYF::template L<5>::SMEM, LYF::template L<6>::SMEM));
  static constexpr int MINB = std::min(std::min(LYF::template L<3>::MINB, LYF::template L<4>::MINB),
                                       std::min(LYF::template L<5>::MINB, LYF::template L<6>::MINB));
};
struct KBQ {
  template <int N> using L = KBLayout<2, N, float, 0>;
};
struct KAQ {
  template <int N> using L = KALayout<2, N, float, 0>;
};

__global__ void __launch_bounds__(GMax<KBQ>::THREADS, GMax<KBQ>::MINB) kb_group(const __grid_constant__ GroupArgs G) {
  const int b = blockIdx.x;
  if (b < G.cum[1]) kb_tensor_body<2, 3, float, 0>(G.a[0], b - G.cum[0]);
  else if (b < G.cum[2]) kb_tensor_body<2, 4, float, 0>(G.a[1], b - G.cum[1]);
  else if (b < G.cum[3]) kb_tensor_body<2, 5, float, 0>(G.a[2], b - G.cum[2]);
  else if (b < G.cum[4]) kb_tensor_body<2, 6, float, 0>(G.a[3], b - G.cum[3]);
}

__global__ void __launch_bounds__(GMax<KAQ>::THREADS, GMax<KAQ>::MINB) ka_group(const __grid_constant__ GroupArgs G) {
  const int b = blockIdx.x;
  if (b < G.cum[1]) ka_tensor_body<2, 3, float, 0>(G.a[0], b - G.cum[0]);
  else if (b < G.cum[2]) ka_tensor_body<2, 4, float, 0>(G.a[1], b - G.cum[1]);
  else if (b < G.cum[3]) ka_tensor_body<2, 5, float, 0>(G.a[2], b - G.cum[2]);
  else if (b < G.cum[4]) ka_tensor_body<2, 6, float, 0>(G.a[3], b - G.cum[3]);
}

template <int N>
constexpr int kb_et() { return KBLayout<2, N, float, 0>::ET; }
template <int N>
constexpr int ka_et() { return KALayout<2, N, float, 0>::ET; }

}  // namespace frp

using namespace frp;

struct fr_group {
  fr_field* f[kGroupMax] = {nullptr, nullptr, nullptr, nullptr};
  GroupArgs gb{}, ga{};
  int nb = 0, na = 0;          // blocks of the kb and ka launches
  cudaStream_t cap = nullptr;
  cudaGraphExec_t g_steps = nullptr, g_step1 = nullptr;
};

namespace {

constexpr int kGroupSteps = 16;

#define GCK(x)                               \
  do {                                       \
    if ((x) != cudaSuccess) return FR_ECUDA; \
  } while (0)

int launch_group_step(fr_group* g, cudaStream_t s) {
  for (int st = 1; st <= 4; ++st) {
    GroupArgs b = g->gb, a = g->ga;
    for (int k = 0; k < kGroupMax; ++k) {
      b.a[k].stage = st;
      a.a[k].stage = st;
    }
    kb_group<<<(unsigned)g->nb, GMax<KBQ>::THREADS, GMax<KBQ>::SMEM, s>>>(b);
    ka_group<<<(unsigned)g->na, GMax<KAQ>::THREADS, GMax<KAQ>::SMEM, s>>>(a);
  }
  GCK(cudaGetLastError());
  return FR_OK;
}

template <typename Body>
int capture(fr_group* g, cudaGraphExec_t* out, Body body) {
  if (!g->cap) GCK(cudaStreamCreateWithFlags(&g->cap, cudaStreamNonBlocking));
  GCK(cudaStreamBeginCapture(g->cap, cudaStreamCaptureModeThreadLocal));
  const int rc = body(g->cap);
  cudaGraph_t gr = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(g->cap, &gr);
  if (rc != FR_OK || ec != cudaSuccess || gr == nullptr) {
    if (gr) cudaGraphDestroy(gr);
    cudaGetLastError();
    return rc != FR_OK ? rc : FR_ECUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(out, gr, 0);
  cudaGraphDestroy(gr);
  if (ei != cudaSuccess) {
    *out = nullptr;
    return FR_ECUDA;
  }
  return FR_OK;
}

// n group steps with no preconditioning due among them
int group_steps(fr_group* g, int n, cudaStream_t s) {
  if (n >= kGroupSteps && !g->g_steps) {
    const int rc = capture(g, &g->g_steps, [g](cudaStream_t c) {
      for (int i = 0; i < kGroupSteps; ++i) {
        const int r = launch_group_step(g, c);
        if (r) return r;
      }
      return (int)FR_OK;
    });
    if (rc) return rc;
  }
  if (n % kGroupSteps && !g->g_step1) {
    const int rc = capture(g, &g->g_step1, [g](cudaStream_t c) { return launch_group_step(g, c); });
    if (rc) return rc;
  }
  for (int i = 0; i < n / kGroupSteps; ++i) GCK(cudaGraphLaunch(g->g_steps, s));
  for (int i = 0; i < n % kGroupSteps; ++i) GCK(cudaGraphLaunch(g->g_step1, s));
  return FR_OK;
}

}  // namespace

extern "C" int fr_group_create(fr_field* const* fields, int n, fr_group** out) {
  if (!fields || !out || n < 1 || n > kGroupMax) return FR_EINVAL;
  *out = nullptr;
  fr_group* g = new (std::nothrow) fr_group();
  if (!g) return FR_ENOMEM;
  for (int i = 0; i < n; ++i) {
    fr_field* f = fields[i];
    if (!f) {
      delete g;
      return FR_EINVAL;
    }
    const int slot = f->order - kGroupPmin;
    if (f->etype != FR_QUAD || f->precision != FR_MIXED || slot < 0 || slot >= kGroupMax || g->f[slot] ||
        f->prm.n_precond != fields[0]->prm.n_precond || f->nstep != fields[0]->nstep) {
      delete g;
      return FR_EUNSUPPORTED;
    }
    g->f[slot] = f;
  }
  static bool prepared = false;
  if (!prepared) {
    if (cudaFuncSetAttribute(kb_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GMax<KBQ>::SMEM) !=
            cudaSuccess ||
        cudaFuncSetAttribute(ka_group, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)GMax<KAQ>::SMEM) !=
            cudaSuccess) {
      delete g;
      return FR_ECUDA;
    }
    prepared = true;
  }
  const int etb[kGroupMax] = {kb_et<3>(), kb_et<4>(), kb_et<5>(), kb_et<6>()};
  const int eta[kGroupMax] = {ka_et<3>(), ka_et<4>(), ka_et<5>(), ka_et<6>()};
  g->gb.cum[0] = g->ga.cum[0] = 0;
  for (int k = 0; k < kGroupMax; ++k) {
    const fr_field* f = g->f[k];
    const int64_t E = f ? f->E : 0;
    g->gb.cum[k + 1] = g->gb.cum[k] + (int)((E + etb[k] - 1) / etb[k]);
    g->ga.cum[k + 1] = g->ga.cum[k] + (int)((E + eta[k] - 1) / eta[k]);
    if (f) {
      KArgs a = f->args;
      a.use_dev_time = 1;
      a.dt = f->prm.dt;
      a.rk = rk_const(a.dt);
      g->gb.a[k] = a;
      g->ga.a[k] = a;
    } else {
      std::memset(&g->gb.a[k], 0, sizeof(KArgs));
      std::memset(&g->ga.a[k], 0, sizeof(KArgs));
    }
  }
  g->nb = g->gb.cum[kGroupMax];
  g->na = g->ga.cum[kGroupMax];
  *out = g;
  return FR_OK;
}

extern "C" int fr_group_step(fr_group* g, int n_steps, void* stream) {
  if (!g || n_steps < 0) return FR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  fr_field* f0 = nullptr;
  for (fr_field* f : g->f)
    if (f && !f0) f0 = f;
  const int64_t np = f0->prm.n_precond;
  int done = 0;
  while (done < n_steps) {
    const int64_t nstep = f0->nstep;
    if (nstep > 0 && nstep % np == 0)
      for (fr_field* f : g->f)
        if (f && f->prm.normal == FR_NORMAL_PSI) {
          const int rc = fr_precondition(f, s);
          if (rc) return rc;
        }
    const int64_t next = (nstep / np + 1) * np;
    const int chunk = (int)std::min<int64_t>(n_steps - done, next - nstep);
    const int rc = group_steps(g, chunk, s);
    if (rc) return rc;
    for (fr_field* f : g->f)
      if (f) f->nstep += chunk;
    done += chunk;
  }
  return FR_OK;
}

extern "C" void fr_group_destroy(fr_group* g) {
  if (!g) return;
  for (cudaGraphExec_t* e : {&g->g_steps, &g->g_step1})
    if (*e) cudaGraphExecDestroy(*e);
  if (g->cap) cudaStreamDestroy(g->cap);
  delete g;
}
