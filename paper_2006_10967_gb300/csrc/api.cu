// C ABI of libfrpcpf: field life cycle, RK4 march, preconditioning schedule,
// mass integral and state transfer.  Device memory is a caller-provided
// workspace; the library never allocates device memory.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "field.cuh"

using namespace frp;

namespace {

constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

struct Layout {
  size_t status, dstate, red, geo, geof, fnbr, wdet, ustg, u, acc, rp, tr, fc, psi0, xfer, vsu, vsf, tacc, wdetf, ep, mcg;
  size_t tri_d, tri_f, tri_high;  // dense triangle operators (double, float), mode mask
  size_t wphys;                   // triangles: physical edge quadrature weight per flux point (float-float)
  size_t ffw;                     // hexahedra: face words (KArgs.ffw)
  size_t total;
};

// number of values in the packed dense triangle operators
size_t tri_op_count(const fr_mesh& m) {
  const size_t NU = m.nu, NF = m.nf;
  return NU * 2 + NF * 2 + NF * 2 + NF * NU + 3 * NU * NU + NU * NF;
}

template <typename R>
void pack_tri(const TriRef& t, std::vector<R>& out) {
  out.clear();
  for (const std::vector<double>* v : {&t.xu, &t.xf, &t.nref, &t.L, &t.Dr, &t.Ds, &t.LIFT, &t.Vinv})
    for (double x : *v) out.push_back((R)x);
}

template <typename R>
TriOpsT<R> tri_pointers(const TriRef& t, const R* base, const uint8_t* high) {
  TriOpsT<R> o;
  const R* p = base;
  o.xu = p; p += t.xu.size();
  o.xf = p; p += t.xf.size();
  o.nref = p; p += t.nref.size();
  o.L = p; p += t.L.size();
  o.Dr = p; p += t.Dr.size();
  o.Ds = p; p += t.Ds.size();
  o.LIFT = p; p += t.LIFT.size();
  o.Vinv = p;
  o.high = high;
  return o;
}

template <typename R>
void fill_vel(const fr_velocity& v, VelDescT<R>& d) {
  std::memset(&d, 0, sizeof(d));
  d.kind = v.kind;
  for (int c = 0; c < 3; ++c) d.a[c] = (R)v.a[c];
  if (v.kind == FR_VEL_STREAM) {
    d.n_modes = v.n_modes;
    for (int k = 0; k < v.n_modes; ++k) {
      d.kx[k] = (R)v.kx[k];
      d.ky[k] = (R)v.ky[k];
      d.A[k] = (R)v.A[k];
      d.B[k] = (R)v.B[k];
    }
  }
}

template <typename R>
void fill_bulk(const fr_params* prm, const fr_mesh* m, BulkConst<R>& b) {
  std::memset(&b, 0, sizeof(b));
  fill_vel<R>(prm->vel, b.vel);
  b.prm.gamma = (R)prm->gamma;
  b.prm.eps = (R)prm->eps;
  b.prm.tau = (R)prm->tau;
  b.prm.tau_psi = (R)prm->tau_psi;
  b.prm.tau_pseudo = (R)prm->tau_pseudo;
  b.prm.delta = (R)prm->delta;
  b.prm.nphi = prm->normal == FR_NORMAL_PHI;
  b.prm.noflux = prm->wall == FR_WALL_NOFLUX;
  if (m->etype != FR_TRI) {
    const Tensor1D& t = m->t1;
    for (int i = 0; i < t.n; ++i) {
      b.ops.x[i] = (R)t.x[i];
      b.ops.w[i] = (R)t.w[i];
      for (int j = 0; j < (m->dim == 2 ? 1 : t.n); ++j) {
        // face weight of face point i + n j: w_i (2D) or w_i w_j (3D)
        const double wf = m->dim == 2 ? t.w[i] : t.w[i] * t.w[j];
        const float hi = (float)wf;
        b.ops.wff[i + t.n * j] = make_float2(hi, (float)(wf - (double)hi));
      }
      b.ops.lend[0][i] = (R)t.lend[0][i];
      b.ops.lend[1][i] = (R)t.lend[1][i];
      b.ops.gLd[i] = (R)t.gLd[i];
      b.ops.gRd[i] = (R)t.gRd[i];
      for (int j = 0; j < t.n; ++j) {
        b.ops.D[i][j] = (R)t.D[i][j];
        b.ops.Vinv[i][j] = (R)t.Vinv[i][j];
      }
    }
  }
}

Layout make_layout(const fr_mesh& m, int precision, int max_blocks, int vel_cache) {
  Layout L{};
  const size_t E = (size_t)m.E, NU = m.nu, NF = m.nf, NG = (size_t)m.dim * m.ncoef;
  const size_t tb = precision == FR_FP64 ? 8 : 4;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align_up(off + bytes);
    return o;
  };
  L.status = take(ST_WORDS * sizeof(int32_t));
  L.dstate = take(DS_WORDS * sizeof(double));
  L.red = take((size_t)(max_blocks + 1) * 2 * sizeof(double));
  L.geo = take(E * NG * sizeof(double));
  L.geof = take(E * NG * sizeof(float));
  L.fnbr = take(E * NF * sizeof(int32_t));
  L.wdet = take(E * NU * sizeof(double));
  L.ustg = take(E * 2 * NU * tb);
  L.u = take(E * 2 * NU * sizeof(double));
  L.acc = take(E * 2 * NU * sizeof(double));
  L.rp = take(E * 2 * NU * tb);
  L.tr = take(E * 2 * NF * tb);
  L.fc = take(E * 2 * NF * tb);
  L.psi0 = take(E * NU * sizeof(double));
  L.xfer = take(E * NU * sizeof(double));
  const bool vc = vel_cache;
  L.vsu = vc ? take(E * m.dim * NU * tb) : 0;
  L.vsf = vc ? take(E * m.dim * NF * tb) : 0;
  L.tacc = take(E * 2 * sizeof(double));
  L.wdetf = take(E * NU * 2 * sizeof(float));
  L.ep = take(E * sizeof(ElemPar));
  L.mcg = m.etype != FR_TRI ? take(E * kMetricRec * tb) : 0;  // per-element metric records
  L.ffw = m.etype == FR_HEX ? take(E * 6 * sizeof(int2)) : 0;
  if (m.etype == FR_TRI) {
    const size_t nops = tri_op_count(m);
    L.tri_d = take(nops * sizeof(double));
    L.tri_f = take(nops * sizeof(float));
    L.tri_high = take(NU);
    L.wphys = take(E * NF * 2 * sizeof(float));
  }
  L.total = off;
  return L;
}

// Hexahedra: the face words of KArgs.ffw (see face_link), derived from the
// per-point connectivity.  FR_EINVAL if the points of a face do not all meet
// one face of one partner, or meet it in an order that is not one of the
// eight symmetries of the face's point grid (face_perm).
int hex_face_words(const fr_mesh& m, std::vector<int32_t>& w) {
  const int N = m.n, NFP = m.nfp, NF = m.nf, NFC = m.nfaces;
  w.assign((size_t)m.E * NFC * 2, 0);
  for (int64_t e = 0; e < m.E; ++e)
    for (int f = 0; f < NFC; ++f) {
      const int64_t base = e * NF + (int64_t)f * NFP;
      const int32_t w0 = m.fnbr[base];
      const int64_t p0 = w0 >> 1;
      const int64_t pe = p0 / NF;
      const int pf = (int)((p0 % NF) / NFP);
      const int32_t isL = w0 & 1;
      const bool wall = p0 == base;
      int found = -1;
      for (int o = 0; o < 8 && found < 0; ++o) {
        bool ok = true;
        for (int q = 0; q < NFP && ok; ++q) {
          const int64_t p = pe * NF + (int64_t)pf * NFP + face_perm(o, q % N, q / N, N);
          ok = m.fnbr[base + q] == (int32_t)((p << 1) | isL);
        }
        if (ok) found = o;
      }
      if (found < 0 || (wall && found != 0)) return FR_EINVAL;
      const int c0 = face_perm(found, 0, 0, N);
      const int ci = face_perm(found, 1, 0, N) - c0, cj = face_perm(found, 0, 1, N) - c0;
      for (int q = 0; q < NFP; ++q)  // face_perm is affine in (i, j) for a fixed o
        if (c0 + ci * (q % N) + cj * (q / N) != face_perm(found, q % N, q / N, N)) return FR_EINVAL;
      w[(e * NFC + f) * 2] = (int32_t)(pe * 2 * NF + (int64_t)pf * NFP + c0);
      w[(e * NFC + f) * 2 + 1] = (isL ? kFwL : 0) | (wall ? kFwWall : 0) | ((ci & 0x3FF) << 2) | ((cj & 0x3FF) << 12);
    }
  return FR_OK;
}

bool get_kernels(const fr_mesh& m, int precision, int variant, KernelSet* ks) {
  if (m.etype == FR_QUAD) return kernels_quad(m.order, precision, m.E, variant, ks);
  if (m.etype == FR_HEX) return kernels_hex(m.order, precision, m.E, variant, ks);
  return kernels_tri(m.order, precision, m.E, variant, ks);
}

// FR_MIXED: triangles 2 (scalar / tensor-core operator applies), quads and
// hexes 4 (default or half tiles of the physical-step residual and update
// kernels); FR_FP64: 1
int variant_count(const fr_mesh& m, int precision) {
  if (precision != FR_MIXED) return 1;
  return m.etype == FR_TRI ? 2 : 4;
}

int check_params(const fr_params* p) {
  if (!p) return FR_EINVAL;
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) return FR_EINVAL;
  if (p->n_precond < 1 || p->pseudo_kmax < 0) return FR_EINVAL;
  if (p->normal != FR_NORMAL_PSI && p->normal != FR_NORMAL_PHI) return FR_EINVAL;
  if (p->wall != FR_WALL_COPY && p->wall != FR_WALL_NOFLUX) return FR_EINVAL;
  if (p->variant < 0) return FR_EINVAL;
  if (p->pseudo_kmax > 0 && !(p->pseudo_dtau > 0.0)) return FR_EINVAL;
  if (p->precision != FR_FP64 && p->precision != FR_MIXED) return FR_EINVAL;
  if (!(p->gamma >= 0.0) || !(p->eps >= 0.0) || !(p->delta > 0.0) || !(p->kappa > 0.0)) return FR_EINVAL;
  if (!(p->nu_max >= 0.0) || !std::isfinite(p->tau) || !std::isfinite(p->tau_psi)) return FR_EINVAL;
  const fr_velocity& v = p->vel;
  if (v.kind < 0 || v.kind > 4) return FR_EINVAL;
  if (v.kind == FR_VEL_STREAM) {
    if (v.n_modes < 1 || v.n_modes > FR_MAX_MODES) return FR_EINVAL;
    if (!v.kx || !v.ky || !v.A || !v.B) return FR_EINVAL;
  }
  return FR_OK;
}

#define CK(x)                                   \
  do {                                          \
    if ((x) != cudaSuccess) return FR_ECUDA;    \
  } while (0)

// ---- small kernels ---------------------------------------------------------
// The solution u is double in the FP64 path and a float-float pair
// (hi, lo) in the mixed path; these helpers read and write one value.
__device__ __forceinline__ double u_get(const KArgs& A, int mixed, int64_t g) {
  if (!mixed) return A.u[g];
  const float2 v = reinterpret_cast<const float2*>(A.u)[g];
  return (double)v.x + (double)v.y;
}
__device__ __forceinline__ void u_put(const KArgs& A, int mixed, int64_t g, double x) {
  if (!mixed) {
    A.u[g] = x;
    return;
  }
  const float hi = (float)x;
  reinterpret_cast<float2*>(A.u)[g] = make_float2(hi, (float)(x - (double)hi));
}

template <typename T>
__global__ void k_reset_psi(KArgs A, int64_t NU, int mixed) {
  const int64_t n = A.E * NU;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / NU, i = g % NU;
    const double p0 = u_get(A, mixed, (e * 2 + 0) * NU + i) - 0.5;
    A.psi0[g] = p0;
    u_put(A, mixed, (e * 2 + 1) * NU + i, p0);
    reinterpret_cast<T*>(A.ustg)[(e * 2 + 1) * NU + i] = (T)p0;
  }
}

template <typename T>
__global__ void k_to_stage(KArgs A, int64_t NU, int mixed) {
  const int64_t n = A.E * 2 * NU;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    reinterpret_cast<T*>(A.ustg)[g] = (T)u_get(A, mixed, g);
}

// field `fld` of u <-> contiguous double buffer
__global__ void k_unpack(KArgs A, int64_t NU, int fld, int mixed, double* out) {
  const int64_t n = A.E * NU;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    out[g] = u_get(A, mixed, (g / NU * 2 + fld) * NU + g % NU);
}
__global__ void k_pack(KArgs A, int64_t NU, int fld, int mixed, const double* in) {
  const int64_t n = A.E * NU;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    u_put(A, mixed, (g / NU * 2 + fld) * NU + g % NU, in[g]);
}

// Neumaier two-term accumulation
__device__ __forceinline__ void neu_add(double& s, double& c, double x) {
  const double t = s + x;
  c += fabs(s) >= fabs(x) ? (s - t) + x : (x - t) + s;
  s = t;
}

// Compensated, fixed-order integral of field `fld` with weights wdet.
__global__ void k_mass(KArgs A, int64_t NU, int fld, int mixed) {
  __shared__ double ss[kThreads], sc[kThreads];
  __shared__ bool last;
  const int64_t n = A.E * NU;
  double s = 0.0, c = 0.0;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / NU, i = g % NU;
    neu_add(s, c, A.wdet[g] * u_get(A, mixed, (e * 2 + fld) * NU + i));
  }
  ss[threadIdx.x] = s;
  sc[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double bs = 0.0, bc = 0.0;
    for (int t = 0; t < (int)blockDim.x; ++t) {
      neu_add(bs, bc, ss[t]);
      bc += sc[t];
    }
    A.red[2 * blockIdx.x] = bs;
    A.red[2 * blockIdx.x + 1] = bc;
    __threadfence();
    last = atomicAdd(&A.status[ST_COUNTER], 1) == (int)gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    __threadfence();
    double ts = 0.0, tc = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      neu_add(ts, tc, ((volatile double*)A.red)[2 * b]);
      tc += ((volatile double*)A.red)[2 * b + 1];
    }
    A.dstate[DS_MASS] = ts + tc;
    A.status[ST_COUNTER] = 0;
  }
}

}  // namespace


namespace {

void launch_elementwise_grid(int64_t n, int* grid) {
  int64_t g = (n + kThreads - 1) / kThreads;
  if (g > 152 * 16) g = 152 * 16;
  if (g < 1) g = 1;
  *grid = (int)g;
}

// Launch one FR kernel; with profiling on, bracket it by CUDA events.
// cls: 0 kb physical, 1 ka physical, 2 kb preconditioning, 3 ka preconditioning
void timed(fr_field* f, int cls, LaunchFn fn, const KArgs& a, cudaStream_t s) {
  if (!f->profiling) {
    fn(a, s);
    return;
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  fn(a, s);
  cudaEventRecord(e1, s);
  f->prof[cls].emplace_back(e0, e1);
}

int stage_and_traces(fr_field* f, cudaStream_t s) {
  int grid;
  launch_elementwise_grid(f->E * 2 * f->nu, &grid);
  if (f->precision == FR_FP64) k_to_stage<double><<<grid, kThreads, 0, s>>>(f->args, f->nu, 0);
  else k_to_stage<float><<<grid, kThreads, 0, s>>>(f->args, f->nu, 1);
  KArgs a = f->args;
  a.stage = 0;
  f->ks.ka[0](a, s);
  CK(cudaGetLastError());
  return FR_OK;
}

// The launch sequence of one preconditioning: reset psi0/psi, traces, then
// k_max pseudo-time RK4 iterations (iterations after the stop rule holds
// exit at once on the device).
int launch_precondition(fr_field* f, cudaStream_t s) {
  CK(cudaMemsetAsync(f->args.status + ST_PSEUDO_DONE, 0, 3 * sizeof(int32_t), s));
  int grid;
  launch_elementwise_grid(f->E * f->nu, &grid);
  if (f->precision == FR_FP64) k_reset_psi<double><<<grid, kThreads, 0, s>>>(f->args, f->nu, 0);
  else k_reset_psi<float><<<grid, kThreads, 0, s>>>(f->args, f->nu, 1);
  KArgs a = f->args;
  a.stage = 0;
  a.dt = f->prm.pseudo_dtau;
  a.rk = rk_const(a.dt);
  a.use_dev_time = 0;
  f->ks.ka[1](a, s);
  for (int k = 0; k < f->prm.pseudo_kmax; ++k)
    for (int st = 1; st <= 4; ++st) {
      a.stage = st;
      timed(f, 2, f->ks.kb[1], a, s);
      timed(f, 3, f->ks.ka[1], a, s);
    }
  CK(cudaGetLastError());
  return FR_OK;
}

// The launch sequence of one physical RK4 step (the time lives on the device).
int launch_rk_step(fr_field* f, cudaStream_t s) {
  KArgs a = f->args;
  a.use_dev_time = 1;
  a.dt = f->prm.dt;
  a.rk = rk_const(a.dt);
  for (int st = 1; st <= 4; ++st) {
    a.stage = st;
    timed(f, 0, f->ks.kb[0], a, s);
    timed(f, 1, f->ks.ka[0], a, s);
  }
  CK(cudaGetLastError());
  return FR_OK;
}

bool graphs_on(const fr_field* f) { return f->use_graphs && !f->profiling; }

// Releases the captured graphs (they hold the launch arguments by value).
void drop_graphs(fr_field* f) {
  for (cudaGraphExec_t* g : {&f->g_steps, &f->g_step1, &f->g_pre})
    if (*g) {
      cudaGraphExecDestroy(*g);
      *g = nullptr;
    }
}

// Records body(stream) on the field's capture stream and instantiates it.
// The launch arguments are fixed for the life of a field, so a graph stays
// valid until the field is destroyed.
template <typename Body>
int capture_graph(fr_field* f, cudaGraphExec_t* out, Body body) {
  if (!f->cap) CK(cudaStreamCreateWithFlags(&f->cap, cudaStreamNonBlocking));
  CK(cudaStreamBeginCapture(f->cap, cudaStreamCaptureModeThreadLocal));
  const int rc = body(f->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(f->cap, &g);
  if (rc != FR_OK || ec != cudaSuccess || g == nullptr) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return rc != FR_OK ? rc : FR_ECUDA;
  }
  const cudaError_t ei = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ei != cudaSuccess) {
    *out = nullptr;
    return FR_ECUDA;
  }
  return FR_OK;
}

int run_precondition(fr_field* f, cudaStream_t s) {
  if (graphs_on(f)) {
    if (!f->g_pre) {
      const int rc = capture_graph(f, &f->g_pre, [f](cudaStream_t c) { return launch_precondition(f, c); });
      if (rc) return rc;
    }
    CK(cudaGraphLaunch(f->g_pre, s));
  } else {
    const int rc = launch_precondition(f, s);
    if (rc) return rc;
  }
  f->n_precond_done++;
  return FR_OK;
}

constexpr int kGraphSteps = 16;  // RK steps per replay of the step graph

// n physical RK steps with no preconditioning due among them.
int launch_rk_steps(fr_field* f, int n, cudaStream_t s) {
  if (!graphs_on(f)) {
    for (int i = 0; i < n; ++i) {
      const int rc = launch_rk_step(f, s);
      if (rc) return rc;
    }
    return FR_OK;
  }
  if (n >= kGraphSteps && !f->g_steps) {
    const int rc = capture_graph(f, &f->g_steps, [f](cudaStream_t c) {
      for (int i = 0; i < kGraphSteps; ++i) {
        const int r = launch_rk_step(f, c);
        if (r) return r;
      }
      return (int)FR_OK;
    });
    if (rc) return rc;
  }
  if (n % kGraphSteps && !f->g_step1) {
    const int rc = capture_graph(f, &f->g_step1, [f](cudaStream_t c) { return launch_rk_step(f, c); });
    if (rc) return rc;
  }
  for (int i = 0; i < n / kGraphSteps; ++i) CK(cudaGraphLaunch(f->g_steps, s));
  for (int i = 0; i < n % kGraphSteps; ++i) CK(cudaGraphLaunch(f->g_step1, s));
  return FR_OK;
}

// n_steps physical steps; a preconditioning runs before every step whose
// index is a positive multiple of n_precond.
int run_steps(fr_field* f, int n_steps, cudaStream_t s) {
  const int64_t np = f->prm.n_precond;
  int done = 0;
  while (done < n_steps) {
    if (f->prm.normal == FR_NORMAL_PSI && f->nstep > 0 && f->nstep % np == 0) {
      const int rc = run_precondition(f, s);
      if (rc) return rc;
    }
    const int64_t next = (f->nstep / np + 1) * np;
    const int chunk = (int)std::min<int64_t>(n_steps - done, next - f->nstep);
    const int rc = launch_rk_steps(f, chunk, s);
    if (rc) return rc;
    f->nstep += chunk;
    done += chunk;
  }
  return FR_OK;
}

int run_step(fr_field* f, cudaStream_t s) { return run_steps(f, 1, s); }

}  // namespace

namespace frp {
int field_run_step(fr_field* f, cudaStream_t s, bool allow_precondition) {
  if (!allow_precondition && f->nstep > 0 && f->nstep % f->prm.n_precond == 0) return FR_EUNSUPPORTED;
  return run_step(f, s);
}
int field_stage_and_traces(fr_field* f, cudaStream_t s) { return stage_and_traces(f, s); }
int field_precondition_begin(fr_field* f, cudaStream_t s) {
  CK(cudaMemsetAsync(f->args.status + ST_PSEUDO_DONE, 0, 3 * sizeof(int32_t), s));
  int grid;
  launch_elementwise_grid(f->E * f->nu, &grid);
  if (f->precision == FR_FP64) k_reset_psi<double><<<grid, kThreads, 0, s>>>(f->args, f->nu, 0);
  else k_reset_psi<float><<<grid, kThreads, 0, s>>>(f->args, f->nu, 1);
  KArgs a = f->args;
  a.stage = 0;
  a.dt = f->prm.pseudo_dtau;
  a.rk = rk_const(a.dt);
  a.use_dev_time = 0;
  f->ks.ka[1](a, s);
  CK(cudaGetLastError());
  return FR_OK;
}
}  // namespace frp

namespace {

int read_status(fr_field* f, cudaStream_t s) {
  int32_t st[ST_WORDS];
  CK(cudaMemcpyAsync(st, f->args.status, sizeof(st), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st[ST_STATUS] != 0 && f->sticky == FR_OK) f->sticky = st[ST_STATUS];
  return f->sticky;
}

}  // namespace

extern "C" int fr_field_workspace_bytes(const fr_mesh* m, const fr_params* prm, size_t* bytes) {
  if (!m || !bytes) return FR_EINVAL;
  int rc = check_params(prm);
  if (rc) return rc;
  KernelSet ks;
  if (!get_kernels(*m, prm->precision, prm->variant, &ks)) return FR_EUNSUPPORTED;
  int mg;
  launch_elementwise_grid(m->E * m->nu, &mg);
  const int mb = ks.max_blocks > mg ? ks.max_blocks : mg;
  *bytes = make_layout(*m, prm->precision, mb, prm->vel_cache).total;
  return FR_OK;
}

extern "C" int fr_field_init(const fr_mesh* m, const fr_params* prm, const fr_ic* ic, void* ws,
                             size_t ws_bytes, void* stream, fr_field** out) {
  if (!m || !ic || !out) return FR_EINVAL;
  *out = nullptr;
  int rc = check_params(prm);
  if (rc) return rc;
  if (!ws || (reinterpret_cast<uintptr_t>(ws) % kAlign) != 0) return FR_EINVAL;
  KernelSet ks;
  if (!get_kernels(*m, prm->precision, prm->variant, &ks)) return FR_EUNSUPPORTED;
  if (!ks.prepared) return FR_ECUDA;
  int mg;
  launch_elementwise_grid(m->E * m->nu, &mg);
  const int mb = ks.max_blocks > mg ? ks.max_blocks : mg;
  const Layout L = make_layout(*m, prm->precision, mb, prm->vel_cache);
  if (ws_bytes < L.total) return FR_ENOMEM;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);

  // initial phi at the solution points
  const int64_t ndof = m->E * m->nu;
  std::vector<double> phi(ndof);
  if (ic->kind == FR_IC_CIRCLE) {
    for (int64_t g = 0; g < ndof; ++g) {
      double r2 = 0.0;
      for (int c = 0; c < m->dim; ++c) {
        const double d = m->xu[g * m->dim + c] - ic->centre[c];
        r2 += d * d;
      }
      phi[g] = 0.5 * (1.0 + std::tanh(ic->beta * (ic->radius - std::sqrt(r2))));
    }
  } else if (ic->kind == FR_IC_ARRAY) {
    if (!ic->phi0) return FR_EINVAL;
    std::memcpy(phi.data(), ic->phi0, ndof * sizeof(double));
  } else {
    return FR_EINVAL;
  }
  for (int64_t g = 0; g < ndof; ++g)
    if (!std::isfinite(phi[g])) return FR_ENONFINITE;
  std::vector<int32_t> ffw;
  if (L.ffw) {
    rc = hex_face_words(*m, ffw);
    if (rc != FR_OK) return rc;
  }

  fr_field* f = new (std::nothrow) fr_field();
  if (!f) return FR_ENOMEM;
  f->dim = m->dim;
  f->etype = m->etype;
  f->order = m->order;
  f->nu = m->nu;
  f->nf = m->nf;
  f->E = m->E;
  f->precision = prm->precision;
  f->prm = *prm;
  f->ks = ks;
  launch_elementwise_grid(ndof, &f->mass_grid);

  char* b = reinterpret_cast<char*>(ws);
  KArgs& A = f->args;
  A.E = m->E;
  A.status = reinterpret_cast<int32_t*>(b + L.status);
  A.dstate = reinterpret_cast<double*>(b + L.dstate);
  A.red = reinterpret_cast<double*>(b + L.red);
  A.geo = reinterpret_cast<const double*>(b + L.geo);
  A.geof = reinterpret_cast<const float*>(b + L.geof);
  A.fnbr = reinterpret_cast<const int32_t*>(b + L.fnbr);
  A.ffw = L.ffw ? reinterpret_cast<const int2*>(b + L.ffw) : nullptr;
  A.wdet = reinterpret_cast<const double*>(b + L.wdet);
  A.ustg = b + L.ustg;
  A.u = reinterpret_cast<double*>(b + L.u);
  A.acc = reinterpret_cast<double*>(b + L.acc);
  A.rp = b + L.rp;
  A.tr = b + L.tr;
  A.fc = b + L.fc;
  A.psi0 = reinterpret_cast<double*>(b + L.psi0);
  f->xfer = reinterpret_cast<double*>(b + L.xfer);
  A.vsu = L.vsu ? b + L.vsu : nullptr;
  A.vsf = L.vsf ? b + L.vsf : nullptr;
  // element flux balances of the mixed path's conservation correction (tensor elements)
  A.tacc = prm->precision == FR_MIXED ? reinterpret_cast<double*>(b + L.tacc) : nullptr;
  A.wphys = m->etype == FR_TRI ? reinterpret_cast<const float2*>(b + L.wphys) : nullptr;
  A.wdetf = reinterpret_cast<const float2*>(b + L.wdetf);
  A.ep = nullptr;
  A.mcg = L.mcg ? b + L.mcg : nullptr;
  f->ep_region = reinterpret_cast<ElemPar*>(b + L.ep);
  A.out = nullptr;
  A.stage = 0;
  A.use_dev_time = 0;
  A.t = 0.0;
  A.dt = prm->dt;
  A.rk = rk_const(prm->dt);
  A.prm.gamma = prm->gamma;
  A.prm.eps = prm->eps;
  A.prm.tau = prm->tau;
  A.prm.tau_psi = prm->tau_psi;
  A.prm.tau_pseudo = prm->tau_pseudo;
  A.prm.delta = prm->delta;
  A.prm.s0 = prm->s0;
  A.prm.kappa = prm->kappa;
  A.prm.nu_max = prm->nu_max;
  A.prm.pseudo_tol = prm->pseudo_tol;
  A.prm.pseudo_fixed = prm->pseudo_fixed;
  A.prm.T = prm->vel.T;
  A.prm.rT = prm->vel.T > 0.0 ? 1.0 / prm->vel.T : 0.0;
  fill_bulk<double>(prm, m, A.cd);
  fill_bulk<float>(prm, m, A.cf);

  int err = FR_OK;
  auto up = [&](size_t off, const void* src, size_t bytes) {
    if (err == FR_OK && cudaMemcpyAsync(b + off, src, bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
      err = FR_ECUDA;
  };
  up(L.geo, m->geo.data(), m->geo.size() * sizeof(double));
  up(L.fnbr, m->fnbr.data(), m->fnbr.size() * sizeof(int32_t));
  if (L.ffw) up(L.ffw, ffw.data(), ffw.size() * sizeof(int32_t));
  up(L.wdet, m->wdet.data(), m->wdet.size() * sizeof(double));
  std::vector<float> wdetf(m->wdet.size() * 2);
  for (size_t g = 0; g < m->wdet.size(); ++g) {
    const float hi = (float)m->wdet[g];
    wdetf[2 * g] = hi;
    wdetf[2 * g + 1] = (float)(m->wdet[g] - (double)hi);
  }
  up(L.wdetf, wdetf.data(), wdetf.size() * sizeof(float));
  std::vector<float> geof(m->geo.begin(), m->geo.end());
  up(L.geof, geof.data(), geof.size() * sizeof(float));
  std::vector<double> trid;
  std::vector<float> trif;
  if (m->etype == FR_TRI) {
    pack_tri(m->tri, trid);
    pack_tri(m->tri, trif);
    up(L.tri_d, trid.data(), trid.size() * sizeof(double));
    up(L.tri_f, trif.data(), trif.size() * sizeof(float));
    up(L.tri_high, m->tri.high.data(), m->tri.high.size());
    const uint8_t* hi = reinterpret_cast<const uint8_t*>(b + L.tri_high);
    A.trid = tri_pointers<double>(m->tri, reinterpret_cast<const double*>(b + L.tri_d), hi);
    A.trif = tri_pointers<float>(m->tri, reinterpret_cast<const float*>(b + L.tri_f), hi);
    // physical quadrature weight of every flux point, w_j |edge| / 2, computed
    // once per edge from the L side's geometry and given bitwise to both
    // sides, so that the element flux balances telescope exactly
    const int n = m->n, NF = m->nf;
    std::vector<double> w1(n), x1(n);
    {
      frp::Tensor1D t;
      frp::build_tensor1d(m->order, t);
      for (int j = 0; j < n; ++j) w1[j] = t.w[j];
    }
    const double V[3][2] = {{-1, -1}, {1, -1}, {-1, 1}};
    std::vector<double> wp(m->E * NF, 0.0);
    for (int64_t e = 0; e < m->E; ++e)
      for (int k = 0; k < NF; ++k) {
        const int32_t w = m->fnbr[e * NF + k];
        if (!(w & 1)) continue;  // R points take the L side's value
        const int ed = k / n, ed1 = (ed + 1) % 3;
        const double* g = &m->geo[e * 2 * 3];
        double dx[2];
        for (int c = 0; c < 2; ++c)
          dx[c] = g[c * 3 + 1] * (V[ed1][0] - V[ed][0]) + g[c * 3 + 2] * (V[ed1][1] - V[ed][1]);
        const double val = w1[k % n] * 0.5 * std::sqrt(dx[0] * dx[0] + dx[1] * dx[1]);
        wp[e * NF + k] = val;
        wp[(int64_t)(w >> 1)] = val;
      }
    std::vector<float> wpf(wp.size() * 2);
    for (size_t g = 0; g < wp.size(); ++g) {
      const float hi = (float)wp[g];
      wpf[2 * g] = hi;
      wpf[2 * g + 1] = (float)(wp[g] - (double)hi);
    }
    up(L.wphys, wpf.data(), wpf.size() * sizeof(float));
  }
  // u = [phi, phi - 1/2] element-major (float-float pairs in the mixed path)
  std::vector<double> u0(m->E * 2 * m->nu);
  for (int64_t e = 0; e < m->E; ++e)
    for (int i = 0; i < m->nu; ++i) {
      u0[(e * 2 + 0) * m->nu + i] = phi[e * m->nu + i];
      u0[(e * 2 + 1) * m->nu + i] = phi[e * m->nu + i] - 0.5;
    }
  if (prm->precision == FR_MIXED) {
    std::vector<float> pairs(u0.size() * 2);
    for (size_t g = 0; g < u0.size(); ++g) {
      const float hi = (float)u0[g];
      pairs[2 * g] = hi;
      pairs[2 * g + 1] = (float)(u0[g] - (double)hi);
    }
    up(L.u, pairs.data(), pairs.size() * sizeof(float));
  } else {
    up(L.u, u0.data(), u0.size() * sizeof(double));
  }
  std::vector<double> p0(ndof);
  for (int64_t g = 0; g < ndof; ++g) p0[g] = phi[g] - 0.5;
  up(L.psi0, p0.data(), p0.size() * sizeof(double));
  if (err == FR_OK && cudaMemsetAsync(b + L.status, 0, ST_WORDS * sizeof(int32_t), s) != cudaSuccess) err = FR_ECUDA;
  if (err == FR_OK && cudaMemsetAsync(b + L.dstate, 0, DS_WORDS * sizeof(double), s) != cudaSuccess) err = FR_ECUDA;
  if (err == FR_OK && cudaMemsetAsync(b + L.acc, 0, m->E * 2 * m->nu * sizeof(double), s) != cudaSuccess) err = FR_ECUDA;
  if (err == FR_OK && cudaMemsetAsync(b + L.fc, 0, L.psi0 - L.fc, s) != cudaSuccess) err = FR_ECUDA;
  if (err == FR_OK && A.mcg) {
    if (!f->ks.mconst) err = FR_EUNSUPPORTED;
    else f->ks.mconst(A, s);
  }
  if (err == FR_OK && A.vsu) {
    if (!f->ks.vcache) err = FR_EUNSUPPORTED;
    else f->ks.vcache(A, s);
  }
  if (err == FR_OK) err = stage_and_traces(f, s);
  if (err == FR_OK && ic->precondition && prm->normal == FR_NORMAL_PSI) err = run_precondition(f, s);
  if (err == FR_OK && cudaStreamSynchronize(s) != cudaSuccess) err = FR_ECUDA;
  if (err == FR_OK && cudaGetLastError() != cudaSuccess) err = FR_ECUDA;
  if (err != FR_OK) {
    fr_field_destroy(f);
    return err;
  }
  err = read_status(f, s);
  *out = f;
  return err;
}

extern "C" int fr_field_init_batch(const fr_mesh* m, const fr_params* prm, int n_inst, const fr_instance* inst,
                                   int precondition, void* ws, size_t ws_bytes, void* stream, fr_field** out) {
  if (!m || !prm || !inst || n_inst < 1 || !out) return FR_EINVAL;
  *out = nullptr;
  if (m->etype == FR_TRI) return FR_EUNSUPPORTED;
  if (!prm->vel_cache) return FR_EINVAL;
  int64_t next = 0;
  for (int i = 0; i < n_inst; ++i) {
    const fr_instance& I = inst[i];
    if (I.elem_begin != next || I.elem_end <= I.elem_begin || I.elem_end > m->E) return FR_EINVAL;
    next = I.elem_end;
    if (!(I.dt > 0.0) || !(I.eps >= 0.0) || !(I.nu_max >= 0.0)) return FR_EINVAL;
    if (prm->pseudo_kmax > 0 && !(I.pseudo_dtau > 0.0)) return FR_EINVAL;
    if (I.vel.T != prm->vel.T || I.ic.kind != FR_IC_CIRCLE) return FR_EINVAL;
    if (I.vel.kind == FR_VEL_STREAM && (I.vel.n_modes < 1 || I.vel.n_modes > FR_MAX_MODES)) return FR_EINVAL;
  }
  if (next != m->E) return FR_EINVAL;
  // initial phi per instance
  const int64_t ndof = m->E * m->nu;
  std::vector<double> phi(ndof);
  for (int i = 0; i < n_inst; ++i) {
    const fr_instance& I = inst[i];
    for (int64_t g = I.elem_begin * m->nu; g < I.elem_end * m->nu; ++g) {
      double r2 = 0.0;
      for (int c = 0; c < m->dim; ++c) {
        const double d = m->xu[g * m->dim + c] - I.ic.centre[c];
        r2 += d * d;
      }
      phi[g] = 0.5 * (1.0 + std::tanh(I.ic.beta * (I.ic.radius - std::sqrt(r2))));
    }
  }
  fr_ic ic{};
  ic.kind = FR_IC_ARRAY;
  ic.precondition = 0;
  ic.phi0 = phi.data();
  fr_field* f = nullptr;
  int rc = fr_field_init(m, prm, &ic, ws, ws_bytes, stream, &f);
  if (rc) return rc;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  std::vector<ElemPar> ep(m->E);
  for (int i = 0; i < n_inst; ++i) {
    const fr_instance& I = inst[i];
    for (int64_t e = I.elem_begin; e < I.elem_end; ++e) {
      ep[e].dt = I.dt;
      ep[e].dtau = I.pseudo_dtau;
      ep[e].t = 0.0;
      ep[e].eps = I.eps;
      ep[e].nu_max = I.nu_max;
      ep[e].rk = rk_const(I.dt);
      ep[e].rkp = rk_const(I.pseudo_dtau > 0.0 ? I.pseudo_dtau : I.dt);
    }
    // this instance's velocity factor at its points
    KArgs a = f->args;
    a.E = I.elem_end - I.elem_begin;
    a.geo = f->args.geo + I.elem_begin * m->dim * m->ncoef;
    const size_t tb = f->precision == FR_FP64 ? 8 : 4;
    a.vsu = reinterpret_cast<const char*>(f->args.vsu) + I.elem_begin * m->dim * m->nu * tb;
    a.vsf = reinterpret_cast<const char*>(f->args.vsf) + I.elem_begin * m->dim * m->nf * tb;
    fill_vel<double>(I.vel, a.cd.vel);
    f->ks.vcache(a, s);
  }
  if (cudaMemcpyAsync(f->ep_region, ep.data(), ep.size() * sizeof(ElemPar), cudaMemcpyHostToDevice, s) !=
      cudaSuccess) {
    fr_field_destroy(f);
    return FR_ECUDA;
  }
  f->args.ep = f->ep_region;
  drop_graphs(f);  // the launch arguments changed
  // the batch's pseudo step for the launch arguments is per element; keep a positive value
  rc = FR_OK;
  if (precondition && prm->normal == FR_NORMAL_PSI) rc = run_precondition(f, s);
  if (rc == FR_OK && cudaStreamSynchronize(s) != cudaSuccess) rc = FR_ECUDA;
  if (rc == FR_OK) rc = read_status(f, s);
  if (rc != FR_OK && rc != FR_ENONFINITE) {
    fr_field_destroy(f);
    return rc;
  }
  *out = f;
  return rc;
}

extern "C" int fr_step(fr_field* f, int n_steps, void* stream) {
  if (!f || n_steps < 0) return FR_EINVAL;
  const int rc = run_steps(f, n_steps, reinterpret_cast<cudaStream_t>(stream));
  if (rc) return rc;
  return f->sticky;
}

extern "C" int fr_precondition(fr_field* f, void* stream) {
  if (!f) return FR_EINVAL;
  return run_precondition(f, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int fr_sync(fr_field* f, void* stream) {
  if (!f) return FR_EINVAL;
  return read_status(f, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int fr_stats_get(fr_field* f, void* stream, fr_stats* out) {
  if (!f || !out) return FR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int32_t st[ST_WORDS];
  double ds[DS_WORDS];
  CK(cudaMemcpyAsync(st, f->args.status, sizeof(st), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(ds, f->args.dstate, sizeof(ds), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (st[ST_STATUS] != 0 && f->sticky == FR_OK) f->sticky = st[ST_STATUS];
  out->n_steps = f->nstep;
  out->t = ds[DS_TIME];
  out->last_pseudo_iters = st[ST_PSEUDO_ITERS];
  out->status = f->sticky;
  out->last_pseudo_rms = ds[DS_PSEUDO_RMS];
  out->n_preconditions = f->n_precond_done;
  return FR_OK;
}

extern "C" int fr_mass_integral(fr_field* f, int which, double* out_host, void* stream) {
  if (!f || !out_host || which < 0 || which > 1) return FR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  k_mass<<<f->mass_grid, kThreads, 0, s>>>(f->args, f->nu, which, f->precision == FR_MIXED);
  CK(cudaGetLastError());
  CK(cudaMemcpyAsync(out_host, f->args.dstate + DS_MASS, sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return FR_OK;
}

namespace {
int copy_field(fr_field* f, int which, void* dst, const void* src, bool to_state, cudaMemcpyKind kind,
               cudaStream_t s) {
  const size_t NU = f->nu, E = f->E;
  if (which == 2) {
    if (to_state) CK(cudaMemcpyAsync(f->args.psi0, src, E * NU * 8, kind, s));
    else CK(cudaMemcpyAsync(dst, f->args.psi0, E * NU * 8, kind, s));
    return FR_OK;
  }
  if (f->precision == FR_FP64) {
    if (to_state)
      CK(cudaMemcpy2DAsync(f->args.u + which * NU, 2 * NU * 8, src, NU * 8, NU * 8, E, kind, s));
    else
      CK(cudaMemcpy2DAsync(dst, NU * 8, f->args.u + which * NU, 2 * NU * 8, NU * 8, E, kind, s));
    return FR_OK;
  }
  int grid;
  launch_elementwise_grid(f->E * f->nu, &grid);
  if (to_state) {
    CK(cudaMemcpyAsync(f->xfer, src, E * NU * 8, kind, s));
    k_pack<<<grid, kThreads, 0, s>>>(f->args, f->nu, which, 1, f->xfer);
  } else {
    k_unpack<<<grid, kThreads, 0, s>>>(f->args, f->nu, which, 1, f->xfer);
    CK(cudaMemcpyAsync(dst, f->xfer, E * NU * 8, kind, s));
  }
  CK(cudaGetLastError());
  return FR_OK;
}
}  // namespace

extern "C" int fr_field_get(fr_field* f, int which, double* host, void* stream) {
  if (!f || !host || which < 0 || which > 2) return FR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = copy_field(f, which, host, nullptr, false, cudaMemcpyDeviceToHost, s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  return FR_OK;
}

extern "C" int fr_field_set(fr_field* f, int which, const double* host, void* stream) {
  if (!f || !host || which < 0 || which > 2) return FR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = copy_field(f, which, nullptr, host, true, cudaMemcpyHostToDevice, s);
  if (rc) return rc;
  if (which < 2) rc = stage_and_traces(f, s);
  if (rc) return rc;
  CK(cudaStreamSynchronize(s));
  return FR_OK;
}

extern "C" int fr_field_get_device(fr_field* f, int which, double* dev, void* stream) {
  if (!f || !dev || which < 0 || which > 2) return FR_EINVAL;
  return copy_field(f, which, dev, nullptr, false, cudaMemcpyDeviceToDevice, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int fr_field_set_device(fr_field* f, int which, const double* dev, void* stream) {
  if (!f || !dev || which < 0 || which > 2) return FR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  int rc = copy_field(f, which, nullptr, dev, true, cudaMemcpyDeviceToDevice, s);
  if (rc) return rc;
  return which < 2 ? stage_and_traces(f, s) : FR_OK;
}

extern "C" int fr_rhs(fr_field* f, double t, double* dev_out, void* stream) {
  if (!f || !dev_out) return FR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  KArgs a = f->args;
  a.use_dev_time = 0;
  a.t = t;
  a.stage = 1;
  a.dt = f->prm.dt;
  a.rk = rk_const(a.dt);
  f->ks.kb[0](a, s);
  a.stage = -1;
  a.out = dev_out;
  f->ks.ka[0](a, s);
  CK(cudaGetLastError());
  return FR_OK;
}

extern "C" int fr_rhs_pseudo(fr_field* f, double* dev_out, void* stream) {
  if (!f || !dev_out) return FR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  CK(cudaMemsetAsync(f->args.status + ST_PSEUDO_DONE, 0, sizeof(int32_t), s));
  KArgs a = f->args;
  a.use_dev_time = 0;
  a.stage = 1;
  a.dt = f->prm.pseudo_dtau;
  a.rk = rk_const(a.dt);
  f->ks.kb[1](a, s);
  a.stage = -1;
  a.out = dev_out;
  f->ks.ka[1](a, s);
  CK(cudaGetLastError());
  return FR_OK;
}

namespace {
// Element rows of the stage values: gather (dst row r = src row elems[r]) or
// scatter (dst row elems[r] = src row r); an index outside [0, E) is skipped
// and recorded in the status word.
template <typename T>
__global__ void k_halo_rows(KArgs A, const int64_t* elems, int64_t n, int row, T* buf, int gather) {
  T* stg = reinterpret_cast<T*>(A.ustg);
  const int64_t total = n * row;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = t / row;
    const int j = (int)(t - r * row);
    const int64_t e = elems[r];
    if (e < 0 || e >= A.E) {
      atomicExch(&A.status[ST_STATUS], FR_EINVAL);
      continue;
    }
    if (gather) buf[t] = stg[e * row + j];
    else stg[e * row + j] = buf[t];
  }
}

int halo_rows(fr_field* f, const int64_t* elems, int64_t n, void* buf, int gather, cudaStream_t s) {
  if (!f || n < 0 || (n > 0 && (!elems || !buf))) return FR_EINVAL;
  if (n == 0) return FR_OK;
  const int row = 2 * f->nu;
  int grid;
  launch_elementwise_grid(n * row, &grid);
  if (f->precision == FR_FP64)
    k_halo_rows<double><<<grid, kThreads, 0, s>>>(f->args, elems, n, row, static_cast<double*>(buf), gather);
  else
    k_halo_rows<float><<<grid, kThreads, 0, s>>>(f->args, elems, n, row, static_cast<float*>(buf), gather);
  CK(cudaGetLastError());
  return FR_OK;
}
}  // namespace

extern "C" int fr_stage(fr_field* f, int stage, void* stream) {
  if (!f || stage < 1 || stage > 4) return FR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  KArgs a = f->args;
  a.use_dev_time = 1;
  a.dt = f->prm.dt;
  a.rk = rk_const(a.dt);
  a.stage = stage;
  f->ks.kb[0](a, s);
  f->ks.ka[0](a, s);
  CK(cudaGetLastError());
  if (stage == 4) f->nstep++;
  return FR_OK;
}

extern "C" int fr_halo_row_bytes(const fr_field* f, size_t* bytes) {
  if (!f || !bytes) return FR_EINVAL;
  *bytes = (size_t)2 * f->nu * (f->precision == FR_FP64 ? 8 : 4);
  return FR_OK;
}

extern "C" int fr_halo_pack(fr_field* f, const int64_t* elems, int64_t n, void* buf, void* stream) {
  return halo_rows(f, elems, n, buf, 1, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int fr_halo_unpack(fr_field* f, const int64_t* elems, int64_t n, const void* buf, void* stream) {
  return halo_rows(f, elems, n, const_cast<void*>(buf), 0, reinterpret_cast<cudaStream_t>(stream));
}

extern "C" int fr_traces(fr_field* f, void* stream) {
  if (!f) return FR_EINVAL;
  KArgs a = f->args;
  a.stage = 0;
  f->ks.ka[0](a, reinterpret_cast<cudaStream_t>(stream));
  CK(cudaGetLastError());
  return FR_OK;
}

// The preconditioning one pseudo stage at a time, for element-partitioned
// runs: the same launches as launch_precondition, with the caller's ghost
// exchange between them.  Only the fixed iteration count: the stop rule's RMS
// would be taken over the rank's local points, ghosts included.
namespace {
int pseudo_check(const fr_field* f) {
  if (!f) return FR_EINVAL;
  if (f->prm.normal != FR_NORMAL_PSI || !f->prm.pseudo_fixed) return FR_EUNSUPPORTED;
  return FR_OK;
}
}  // namespace

extern "C" int fr_pseudo_begin(fr_field* f, void* stream) {
  int rc = pseudo_check(f);
  if (rc) return rc;
  rc = field_precondition_begin(f, reinterpret_cast<cudaStream_t>(stream));
  if (rc) return rc;
  f->n_precond_done++;
  return FR_OK;
}

extern "C" int fr_pseudo_stage(fr_field* f, int stage, void* stream) {
  const int rc = pseudo_check(f);
  if (rc) return rc;
  if (stage < 1 || stage > 4) return FR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  KArgs a = f->args;
  a.stage = stage;
  a.dt = f->prm.pseudo_dtau;
  a.rk = rk_const(a.dt);
  a.use_dev_time = 0;
  f->ks.kb[1](a, s);
  f->ks.ka[1](a, s);
  CK(cudaGetLastError());
  return FR_OK;
}

extern "C" int fr_kernel_variants(const fr_mesh* m, int precision, int32_t* count) {
  if (!m || !count || (precision != FR_FP64 && precision != FR_MIXED)) return FR_EINVAL;
  *count = variant_count(*m, precision);
  return FR_OK;
}

extern "C" int fr_profile(fr_field* f, int enable) {
  if (!f) return FR_EINVAL;
  f->profiling = enable ? 1 : 0;
  return FR_OK;
}

extern "C" int fr_profile_read(fr_field* f, void* stream, double* total_ms, int64_t* launches) {
  if (!f || !total_ms || !launches) return FR_EINVAL;
  CK(cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream)));
  for (int c = 0; c < 4; ++c) {
    double tot = 0.0;
    for (auto& pr : f->prof[c]) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) != cudaSuccess) return FR_ECUDA;
      tot += ms;
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    total_ms[c] = tot;
    launches[c] = (int64_t)f->prof[c].size();
    f->prof[c].clear();
  }
  return FR_OK;
}

extern "C" int fr_profile_kernel(fr_field* f, int kernel, int n, void* stream, double* ms_per_launch) {
  if (!f || !ms_per_launch || kernel != 0 || n < 1) return FR_EINVAL;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  KArgs a = f->args;
  a.use_dev_time = 1;
  a.dt = f->prm.dt;
  a.rk = rk_const(a.dt);
  a.stage = 1;
  cudaGraphExec_t ge = nullptr;
  int rc = capture_graph(f, &ge, [&](cudaStream_t c) {
    for (int i = 0; i < n; ++i) f->ks.kb[0](a, c);
    CK(cudaGetLastError());
    return (int)FR_OK;
  });
  if (rc) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  float ms = 0.f;
  rc = FR_ECUDA;
  if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
      cudaGraphLaunch(ge, s) == cudaSuccess && cudaEventRecord(e0, s) == cudaSuccess &&
      cudaGraphLaunch(ge, s) == cudaSuccess && cudaEventRecord(e1, s) == cudaSuccess &&
      cudaEventSynchronize(e1) == cudaSuccess && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) {
    *ms_per_launch = (double)ms / n;
    rc = FR_OK;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaGraphExecDestroy(ge);
  return rc;
}

extern "C" void fr_field_destroy(fr_field* f) {
  if (!f) return;
  drop_graphs(f);
  if (f->cap) cudaStreamDestroy(f->cap);
  for (int c = 0; c < 4; ++c)
    for (auto& pr : f->prof[c]) {
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
  delete f;
}

extern "C" const char* fr_strerror(int code) {
  switch (code) {
    case FR_OK: return "ok";
    case FR_EINVAL: return "invalid argument";
    case FR_ENOMEM: return "out of memory or workspace too small";
    case FR_ECUDA: return "CUDA runtime error";
    case FR_ENONFINITE: return "non-finite value in the state";
    case FR_ETIMEOUT: return "bounded device wait timed out";
    case FR_EUNSUPPORTED: return "element type, order or mode not supported";
    case FR_EBOUNDS: return "partner index out of range (bounds-checked build)";
    default: return "unknown error";
  }
}

extern "C" int fr_version(void) { return 100; }
