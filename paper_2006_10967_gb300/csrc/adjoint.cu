// Hand-written discrete adjoint of the FR-PCPF march (C ABI:
// fr_adjoint_workspace_bytes, fr_adjoint_record, fr_adjoint_step).
//
// fr_adjoint_record runs the forward march from the current state and keeps
// the solution every ckpt_every steps in the caller's workspace.
// fr_adjoint_step sweeps backwards: per checkpoint segment it recomputes the
// forward steps, keeping the four RK stage inputs of each step, then applies
// the transpose of each RK4 step,
//   lam_k4 = dt/6 lam'          a4 = (dR/du)^T(U4) lam_k4
//   lam_k3 = dt/3 lam' + dt a4  a3 = (dR/du)^T(U3) lam_k3
//   lam_k2 = dt/3 lam' + dt/2 a3, a2 ...   lam_k1 = dt/6 lam' + dt/2 a2, a1 ...
//   lam = lam' + a4 + a3 + a2 + a1,
// with the vector-Jacobian products of kadj.cuh, and accumulates the
// gradient with respect to the stream-function coefficients.
//
// With FR_ADJ_PRECONDITION the window starts with the t = 0 preconditioning
// (psi0 = psi = phi0 - 1/2, then the fixed count of pseudo-time RK4
// iterations), recorded stage by stage; fr_adjoint_step then continues the
// reverse sweep through the pseudo iterations (adj_b<.., 1>, the same RK4
// recurrence with the pseudo step) and returns dJ/dphi0 along both paths:
// phi0 itself and psi = P(phi0 - 1/2; psi0 = phi0 - 1/2).
//
// Mixed-precision fields: the recorded march is the field's own FP32 one
// (its float-float states are the checkpoints); each segment is recomputed
// from its checkpoint, widened to FP64, by the FP64 kernels on FP64 shadow
// arrays in the workspace, and the sweep linearises along that recomputation
// (velocity evaluated analytically).  Linearising along the FP32 stage inputs
// themselves is ill-conditioned: where phi is small but not zero, psi = phi
// - 1/2 rounded to float has an exactly flat gradient, and the derivative of
// the normal q / max(|q|, delta) there is 1 / delta.  With a preconditioning
// in the window its pseudo iterations are likewise re-run in FP64 from the
// same phi0.  The result is the FP64 scheme's gradient along trajectories
// restarted every ckpt_every steps from the FP32 march.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "field.cuh"
#include "kadj.cuh"
#include "kadj_tri.cuh"
#include "kdispatch.hpp"

using namespace frp;

namespace {

#define CK(x)                                \
  do {                                       \
    if ((x) != cudaSuccess) return FR_ECUDA; \
  } while (0)

size_t al(size_t x) { return (x + 255) / 256 * 256; }

typedef void (*AdjFn)(const AdjArgs&, cudaStream_t);
typedef void (*TabFn)(const KArgs&, double*, cudaStream_t);
struct AdjSet {
  AdjFn a = nullptr, b = nullptr, c = nullptr, b1 = nullptr;  // b1: the preconditioning system
  TabFn tab = nullptr;  // cos/sin table of the stream-function modes at the points
  int et = 1;
};

template <int DIM, int N>
void la(const AdjArgs& B, cudaStream_t s) {
  using LY = AdjLayout<DIM, N>;
  adj_a<DIM, N><<<(unsigned)((B.K.E + LY::ET - 1) / LY::ET), LY::THREADS, 0, s>>>(B);
}
template <int DIM, int N, int MODE>
void lb(const AdjArgs& B, cudaStream_t s) {
  using LY = AdjLayout<DIM, N>;
  static bool init = false;
  if (!init) {
    cudaFuncSetAttribute(adj_b<DIM, N, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LY::SMEM);
    init = true;
  }
  adj_b<DIM, N, MODE><<<(unsigned)((B.K.E + LY::ET - 1) / LY::ET), LY::THREADS, LY::SMEM, s>>>(B);
}
template <int DIM, int N>
void lc(const AdjArgs& B, cudaStream_t s) {
  using LY = AdjLayout<DIM, N>;
  adj_c<DIM, N><<<(unsigned)((B.K.E + LY::ET - 1) / LY::ET), LY::THREADS, 0, s>>>(B);
}
template <int DIM, int N>
void ltab(const KArgs& A, double* cs, cudaStream_t s) {
  const int64_t n = A.E * (TS<DIM, N>::NU + TS<DIM, N>::NF);
  const int64_t g = (n + 255) / 256;
  k_coef_table<DIM, N><<<(unsigned)(g < 152 * 16 ? g : 152 * 16), 256, 0, s>>>(A, cs);
}
template <int DIM, int N>
AdjSet make_set() {
  AdjSet a;
  a.a = la<DIM, N>;
  a.b = lb<DIM, N, 0>;
  a.b1 = lb<DIM, N, 1>;
  a.c = lc<DIM, N>;
  a.tab = ltab<DIM, N>;
  a.et = AdjLayout<DIM, N>::ET;
  return a;
}

// triangles (kadj_tri.cuh)
template <typename K>
void set_smem(K kern, size_t bytes) {
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}
template <int P>
void la_tri(const AdjArgs& B, cudaStream_t s) {
  using LY = AdjTriLayout<P>;
  static bool init = false;
  if (!init) {
    set_smem(adj_a_tri<P>, LY::SMEM);
    init = true;
  }
  adj_a_tri<P><<<(unsigned)((B.K.E + LY::ET - 1) / LY::ET), LY::THREADS, LY::SMEM, s>>>(B);
}
template <int P, int MODE>
void lb_tri(const AdjArgs& B, cudaStream_t s) {
  using LY = AdjTriLayout<P>;
  static bool init = false;
  if (!init) {
    set_smem(adj_b_tri<P, MODE>, LY::SMEM);
    init = true;
  }
  adj_b_tri<P, MODE><<<(unsigned)((B.K.E + LY::ET - 1) / LY::ET), LY::THREADS, LY::SMEM, s>>>(B);
}
template <int P>
void lc_tri(const AdjArgs& B, cudaStream_t s) {
  using LY = AdjTriLayout<P>;
  static bool init = false;
  if (!init) {
    set_smem(adj_c_tri<P>, LY::SMEM);
    init = true;
  }
  adj_c_tri<P><<<(unsigned)((B.K.E + LY::ET - 1) / LY::ET), LY::THREADS, LY::SMEM, s>>>(B);
}
template <int P>
void ltab_tri(const KArgs& A, double* cs, cudaStream_t s) {
  const int64_t n = A.E * (TriS<P>::NU + TriS<P>::NF);
  const int64_t g = (n + 255) / 256;
  k_coef_table_tri<P><<<(unsigned)(g < 152 * 16 ? g : 152 * 16), 256, 0, s>>>(A, cs);
}
template <int P>
AdjSet make_set_tri() {
  AdjSet a;
  a.a = la_tri<P>;
  a.b = lb_tri<P, 0>;
  a.c = lc_tri<P>;
  a.b1 = lb_tri<P, 1>;
  a.tab = ltab_tri<P>;
  a.et = AdjTriLayout<P>::ET;
  return a;
}

bool adj_kernels(const fr_field* f, AdjSet* out) {
  if (f->etype == FR_TRI) {
    switch (f->order) {
      case 1: *out = make_set_tri<1>(); return true;
      case 2: *out = make_set_tri<2>(); return true;
      case 3: *out = make_set_tri<3>(); return true;
      case 4: *out = make_set_tri<4>(); return true;
      case 5: *out = make_set_tri<5>(); return true;
    }
    return false;
  }
  if (f->etype == FR_QUAD) {
    switch (f->order) {
      case 1: *out = make_set<2, 2>(); return true;
      case 2: *out = make_set<2, 3>(); return true;
      case 3: *out = make_set<2, 4>(); return true;
      case 4: *out = make_set<2, 5>(); return true;
      case 5: *out = make_set<2, 6>(); return true;
      case 6: *out = make_set<2, 7>(); return true;
    }
  }
  if (f->etype == FR_HEX) {
    switch (f->order) {
      case 1: *out = make_set<3, 2>(); return true;
      case 2: *out = make_set<3, 3>(); return true;
      case 3: *out = make_set<3, 4>(); return true;
    }
  }
  return false;
}

__global__ void k_pack_lam(double* L, const double* dphi, const double* dpsi, int64_t E, int NU) {
  const int64_t n = E * NU;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / NU, i = g % NU;
    L[(e * 2 + 0) * NU + i] = dphi[g];
    L[(e * 2 + 1) * NU + i] = dpsi ? dpsi[g] : 0.0;
  }
}

__global__ void k_unpack_lam(const double* L, double* out, int64_t E, int NU) {
  const int64_t n = E * NU;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / NU, i = g % NU;
    out[g] = L[(e * 2 + 0) * NU + i];
    out[n + g] = L[(e * 2 + 1) * NU + i];
  }
}

// float-float states widened to FP64 (mixed fields)
__global__ void k_ff_widen(const float2* in, double* out, int64_t n) {
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x)
    out[g] = (double)in[g].x + (double)in[g].y;
}

// psi0 = psi = phi - 1/2 on the FP64 shadow (the start of its preconditioning)
__global__ void k_reset_psi64(KArgs A, int64_t NU) {
  const int64_t n = A.E * NU;
  double* st = reinterpret_cast<double*>(A.ustg);
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / NU, i = g % NU;
    const double p0 = A.u[(e * 2 + 0) * NU + i] - 0.5;
    A.psi0[g] = p0;
    A.u[(e * 2 + 1) * NU + i] = p0;
    st[(e * 2 + 1) * NU + i] = p0;
  }
}

// The FP64 shadow of a mixed field's arguments (workspace arrays; velocity
// evaluated analytically)
KArgs shadow_args(const fr_field* f, const AdjRecord& R) {
  KArgs a = f->args;
  a.u = reinterpret_cast<double*>(R.ws + R.off_u64);
  a.ustg = R.ws + R.off_stg64;
  a.acc = reinterpret_cast<double*>(R.ws + R.off_acc64);
  a.rp = R.ws + R.off_rp64;
  a.tr = R.ws + R.off_trd;
  a.fc = R.ws + R.off_fc64;
  a.mcg = R.ws + R.off_mc64;
  a.vsu = a.vsf = nullptr;
  a.tacc = nullptr;
  a.ep = nullptr;
  return a;
}

// The FP64 kernel set of the field's element type and order (the traces of
// the widened stage inputs of a mixed field).
bool fp64_kernels(const fr_field* f, KernelSet* ks) {
  if (f->etype == FR_QUAD) return kernels_quad(f->order, FR_FP64, f->E, 0, ks);
  if (f->etype == FR_HEX) return kernels_hex(f->order, FR_FP64, f->E, 0, ks);
  if (f->etype == FR_TRI) return kernels_tri(f->order, FR_FP64, f->E, 0, ks);
  return false;
}

// preconditioning sweep: keep phi's adjoint (out[0..n)) and zero it in L
__global__ void k_zero_phi(double* L, int64_t E, int NU) {
  const int64_t n = E * NU;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / NU, i = g % NU;
    L[(e * 2 + 0) * NU + i] = 0.0;
  }
}

// dJ/dphi0 = lam_phi + lam_psi(start of the pseudo iterations) + lam_psi0;
// psi is no independent input then (its slot of out is zeroed)
__global__ void k_precond_out(double* out, const double* L, const double* lpsi0, int64_t E, int NU) {
  const int64_t n = E * NU;
  for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < n; g += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = g / NU, i = g % NU;
    out[g] += L[(e * 2 + 1) * NU + i] + lpsi0[g];
    out[n + g] = 0.0;
  }
}

// out[m] = sum over blocks of coefp[b][m], in block order
__global__ void k_coef_reduce(const double* coefp, int nblocks, int M2, double* out) {
  const int m = blockIdx.x * blockDim.x + threadIdx.x;
  if (m >= M2) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += coefp[(int64_t)b * M2 + m];
  out[m] = s;
}

struct Sizes {
  size_t ckpt_slot, stage_slot, total;
  int n_ckpt;
};

Sizes sizes(const fr_field* f, int n_steps, int ck, int adj_blocks, int flags) {
  Sizes z;
  const size_t ndof = (size_t)f->E * f->nu;
  z.n_ckpt = (n_steps + ck - 1) / ck;
  z.ckpt_slot = al(2 * ndof * 8 + 8);
  z.stage_slot = al(2 * ndof * 8);
  const size_t nf2 = (size_t)f->E * 2 * f->nf * 8;
  size_t t = 0;
  t += (z.n_ckpt + 1) * z.ckpt_slot;
  t += (size_t)ck * 4 * z.stage_slot;
  t += al((size_t)ck * 8);
  t += 2 * al(nf2);
  t += 4 * al(2 * ndof * 8);
  t += al((size_t)adj_blocks * 2 * FR_MAX_MODES * 8);
  if (f->precision == FR_MIXED)  // FP64 shadow: traces, common flux, state, stage, accumulator, divergence, records
    t += 2 * al(nf2) + 4 * al(2 * ndof * 8) + al((size_t)f->E * kMetricRec * 8);
  if (flags & FR_ADJ_PRECONDITION) {           // pseudo stage inputs, dR_p/dpsi0 adjoint
    t += (size_t)f->prm.pseudo_kmax * 4 * z.stage_slot;
    t += al(ndof * 8);
  }
  if (f->prm.vel.kind == FR_VEL_STREAM) {  // phase table and per-point velocity adjoint
    const size_t np = (size_t)f->E * (f->nu + f->nf);
    t += al(np * (size_t)f->prm.vel.n_modes * 2 * 8);
    t += al(np * 2 * 8);
  }
  z.total = t;
  return z;
}

}  // namespace

extern "C" int fr_adjoint_workspace_bytes(fr_field* f, int n_steps, int ckpt_every, int flags, size_t* bytes) {
  if (!f || !bytes || n_steps < 1 || ckpt_every < 1 || (flags & ~FR_ADJ_PRECONDITION)) return FR_EINVAL;
  AdjSet as;
  if (!adj_kernels(f, &as)) return FR_EUNSUPPORTED;
  const int nb = (int)((f->E + as.et - 1) / as.et);
  *bytes = sizes(f, n_steps, ckpt_every, nb, flags).total;
  return FR_OK;
}

extern "C" int fr_adjoint_record(fr_field* f, int n_steps, int ckpt_every, int flags, void* ws, size_t ws_bytes,
                                 void* stream) {
  if (!f || !ws || n_steps < 1 || ckpt_every < 1 || (flags & ~FR_ADJ_PRECONDITION)) return FR_EINVAL;
  const bool pre = (flags & FR_ADJ_PRECONDITION) != 0;
  // the preconditioning is differentiated for its fixed iteration count
  if (pre && !f->prm.pseudo_fixed) return FR_EUNSUPPORTED;
  if (reinterpret_cast<uintptr_t>(ws) % 256) return FR_EINVAL;
  if (f->prm.normal != FR_NORMAL_PSI) return FR_EUNSUPPORTED;  // adjoint of the preconditioned method only
  if (f->prm.wall != FR_WALL_COPY) return FR_EUNSUPPORTED;     // and of the paper's copy-ghost walls
  if (f->args.ep) return FR_EUNSUPPORTED;                       // one uniform time step (no batch fields)
  AdjSet as;
  if (!adj_kernels(f, &as)) return FR_EUNSUPPORTED;
  const int nb = (int)((f->E + as.et - 1) / as.et);
  const Sizes z = sizes(f, n_steps, ckpt_every, nb, flags);
  if (ws_bytes < z.total) return FR_ENOMEM;
  // the recorded window must not contain a preconditioning step
  for (int64_t n = f->nstep; n < f->nstep + n_steps; ++n)
    if (n > 0 && n % f->prm.n_precond == 0) return FR_EUNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  AdjRecord& R = f->rec;
  R = AdjRecord();
  R.n_steps = n_steps;
  R.ckpt_every = ckpt_every;
  R.n_ckpt = z.n_ckpt;
  R.step0 = f->nstep;
  R.ws = reinterpret_cast<char*>(ws);
  R.bytes = ws_bytes;
  R.adj_blocks = nb;
  size_t off = 0;
  R.off_ckpt = off;
  off += (z.n_ckpt + 1) * z.ckpt_slot;
  R.off_stage = off;
  off += (size_t)ckpt_every * 4 * z.stage_slot;
  R.off_times = off;
  off += al((size_t)ckpt_every * 8);
  const size_t nf2 = al((size_t)f->E * 2 * f->nf * 8), nd2 = al(2 * (size_t)f->E * f->nu * 8);
  R.off_Y = off;
  off += nf2;
  R.off_lamuo = off;
  off += nf2;
  R.off_lamU = off;
  off += nd2;
  R.off_Lp = off;
  off += nd2;
  R.off_Lu = off;
  off += nd2;
  R.off_Lk = off;
  off += nd2;
  R.off_coefp = off;
  off += al((size_t)nb * 2 * FR_MAX_MODES * 8);
  if (f->precision == FR_MIXED) {
    R.off_trd = off;
    off += nf2;
    R.off_fc64 = off;
    off += nf2;
    R.off_u64 = off;
    off += nd2;
    R.off_stg64 = off;
    off += nd2;
    R.off_acc64 = off;
    off += nd2;
    R.off_rp64 = off;
    off += nd2;
    R.off_mc64 = off;
    off += al((size_t)f->E * kMetricRec * 8);
  }
  if (pre) {
    R.precond = 1;
    R.n_pseudo = f->prm.pseudo_kmax;
    R.off_pstage = off;
    off += (size_t)R.n_pseudo * 4 * z.stage_slot;
    R.off_lpsi0 = off;
    off += al((size_t)f->E * f->nu * 8);
  }
  if (f->prm.vel.kind == FR_VEL_STREAM) {
    const size_t np = (size_t)f->E * (f->nu + f->nf);
    R.off_cs = off;
    off += al(np * (size_t)f->prm.vel.n_modes * 2 * 8);
    R.off_lv = off;
  }
  const size_t ubytes = 2 * (size_t)f->E * f->nu * 8;
  const bool mixed = f->precision == FR_MIXED;
  KernelSet ks64{};
  if (mixed && !fp64_kernels(f, &ks64)) return FR_EUNSUPPORTED;
  const int64_t nv = 2 * f->E * f->nu;
  const int grid = (int)std::min<int64_t>((nv + 255) / 256, 152 * 16);
  if (mixed && ks64.mconst) ks64.mconst(shadow_args(f, R), s);  // FP64 metric records of the shadow
  if (pre) {
    // the t = 0 preconditioning, keeping every pseudo stage input (a mixed
    // field's FP32 preconditioning is re-run in FP64 from the same phi0)
    if (mixed)
      k_ff_widen<<<grid, 256, 0, s>>>(reinterpret_cast<const float2*>(f->args.u), reinterpret_cast<double*>(R.ws + R.off_u64), nv);
    int rc = field_precondition_begin(f, s);
    if (rc) return rc;
    KArgs a = f->args;
    a.dt = f->prm.pseudo_dtau;
    a.rk = rk_const(a.dt);
    a.use_dev_time = 0;
    for (int k = 0; k < R.n_pseudo; ++k)
      for (int st = 1; st <= 4; ++st) {
        if (!mixed) {
          char* U = R.ws + R.off_pstage + ((size_t)k * 4 + (st - 1)) * z.stage_slot;
          CK(cudaMemcpyAsync(U, f->args.ustg, ubytes, cudaMemcpyDeviceToDevice, s));
        }
        a.stage = st;
        f->ks.kb[1](a, s);
        f->ks.ka[1](a, s);
      }
    if (mixed) {
      KArgs b = shadow_args(f, R);
      b.dt = f->prm.pseudo_dtau;
      b.rk = rk_const(b.dt);
      b.use_dev_time = 0;
      CK(cudaMemsetAsync(f->args.status + ST_PSEUDO_DONE, 0, 3 * sizeof(int32_t), s));
      k_reset_psi64<<<grid, 256, 0, s>>>(b, f->nu);
      b.stage = 0;
      ks64.ka[1](b, s);
      for (int k = 0; k < R.n_pseudo; ++k)
        for (int st = 1; st <= 4; ++st) {
          char* U = R.ws + R.off_pstage + ((size_t)k * 4 + (st - 1)) * z.stage_slot;
          CK(cudaMemcpyAsync(U, b.ustg, ubytes, cudaMemcpyDeviceToDevice, s));
          b.stage = st;
          ks64.kb[1](b, s);
          ks64.ka[1](b, s);
        }
      CK(cudaMemsetAsync(f->args.status + ST_PSEUDO_DONE, 0, 3 * sizeof(int32_t), s));
    }
    CK(cudaGetLastError());
    f->n_precond_done++;
  }
  for (int n = 0; n < n_steps; ++n) {
    if (n % ckpt_every == 0) {
      char* slot = R.ws + R.off_ckpt + (size_t)(n / ckpt_every) * z.ckpt_slot;
      CK(cudaMemcpyAsync(slot, f->args.u, ubytes, cudaMemcpyDeviceToDevice, s));
      CK(cudaMemcpyAsync(slot + ubytes, f->args.dstate + DS_TIME, 8, cudaMemcpyDeviceToDevice, s));
    }
    const int rc = field_run_step(f, s, false);
    if (rc) return rc;
  }
  char* last = R.ws + R.off_ckpt + (size_t)z.n_ckpt * z.ckpt_slot;
  CK(cudaMemcpyAsync(last, f->args.u, ubytes, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(last + ubytes, f->args.dstate + DS_TIME, 8, cudaMemcpyDeviceToDevice, s));
  R.active = 1;
  return FR_OK;
}

extern "C" int fr_adjoint_step(fr_field* f, const double* dJ_dphiT, const double* dJ_dpsiT, double* dJ_du0,
                               double* dJ_dcoef, void* stream) {
  if (!f || !dJ_dphiT || !dJ_du0) return FR_EINVAL;
  AdjRecord& R = f->rec;
  if (!R.active) return FR_EINVAL;
  AdjSet as;
  if (!adj_kernels(f, &as)) return FR_EUNSUPPORTED;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const bool mixed = f->precision == FR_MIXED;
  KernelSet ks64{};
  if (mixed && !fp64_kernels(f, &ks64)) return FR_EUNSUPPORTED;
  const Sizes z = sizes(f, R.n_steps, R.ckpt_every, R.adj_blocks, R.precond ? FR_ADJ_PRECONDITION : 0);
  const int64_t E = f->E;
  const int NU = f->nu;
  const size_t ubytes = 2 * (size_t)E * NU * 8;
  double* Y = reinterpret_cast<double*>(R.ws + R.off_Y);
  double* lamuo = reinterpret_cast<double*>(R.ws + R.off_lamuo);
  double* lamU = reinterpret_cast<double*>(R.ws + R.off_lamU);
  double* Lp = reinterpret_cast<double*>(R.ws + R.off_Lp);
  double* Lu = reinterpret_cast<double*>(R.ws + R.off_Lu);
  double* Lk = reinterpret_cast<double*>(R.ws + R.off_Lk);
  double* coefp = reinterpret_cast<double*>(R.ws + R.off_coefp);
  double* times = reinterpret_cast<double*>(R.ws + R.off_times);
  const int M2 = f->prm.vel.kind == FR_VEL_STREAM ? 2 * f->args.cd.vel.n_modes : 0;
  const double dt = f->prm.dt;
  int grid = (int)((E * NU + 255) / 256);
  if (grid > 152 * 16) grid = 152 * 16;
  k_pack_lam<<<grid, 256, 0, s>>>(Lp, dJ_dphiT, dJ_dpsiT, E, NU);
  if (M2) CK(cudaMemsetAsync(coefp, 0, (size_t)R.adj_blocks * M2 * 8, s));
  double* cs = M2 ? reinterpret_cast<double*>(R.ws + R.off_cs) : nullptr;
  double* lv = M2 ? reinterpret_cast<double*>(R.ws + R.off_lv) : nullptr;
  if (M2) as.tab(f->args, cs, s);
  const int64_t npts = E * (f->nu + f->nf);
  const int64_t nstep_save = f->nstep;
  std::vector<double> th(R.ckpt_every);
  for (int seg = R.n_ckpt - 1; seg >= 0; --seg) {
    const int s0 = seg * R.ckpt_every;
    const int s1 = s0 + R.ckpt_every < R.n_steps ? s0 + R.ckpt_every : R.n_steps;
    // restore the checkpoint and recompute the segment, keeping the stage inputs
    char* slot = R.ws + R.off_ckpt + (size_t)seg * z.ckpt_slot;
    CK(cudaMemcpyAsync(f->args.dstate + DS_TIME, slot + ubytes, 8, cudaMemcpyDeviceToDevice, s));
    KArgs a = mixed ? shadow_args(f, R) : f->args;
    const KernelSet& ksr = mixed ? ks64 : f->ks;
    if (mixed) {
      // the FP64 shadow from the widened float-float checkpoint
      k_ff_widen<<<grid, 256, 0, s>>>(reinterpret_cast<const float2*>(slot), a.u, 2 * E * NU);
      CK(cudaMemcpyAsync(a.ustg, a.u, ubytes, cudaMemcpyDeviceToDevice, s));
      KArgs b = a;
      b.stage = 0;
      ks64.ka[0](b, s);
    } else {
      CK(cudaMemcpyAsync(f->args.u, slot, ubytes, cudaMemcpyDeviceToDevice, s));
      int rc = field_stage_and_traces(f, s);
      if (rc) return rc;
    }
    f->nstep = R.step0 + s0;
    for (int n = s0; n < s1; ++n) {
      CK(cudaMemcpyAsync(times + (n - s0), f->args.dstate + DS_TIME, 8, cudaMemcpyDeviceToDevice, s));
      a.use_dev_time = 1;
      a.dt = dt;
      a.rk = rk_const(dt);
      for (int st = 1; st <= 4; ++st) {
        char* U = R.ws + R.off_stage + ((size_t)(n - s0) * 4 + (st - 1)) * z.stage_slot;
        CK(cudaMemcpyAsync(U, a.ustg, ubytes, cudaMemcpyDeviceToDevice, s));
        a.stage = st;
        ksr.kb[0](a, s);
        ksr.ka[0](a, s);
      }
      f->nstep++;
    }
    CK(cudaMemcpyAsync(th.data(), times, (size_t)(s1 - s0) * 8, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    // reverse through the segment
    for (int n = s1 - 1; n >= s0; --n) {
      for (int st = 4; st >= 1; --st) {
        AdjArgs B;
        std::memset(&B, 0, sizeof(B));
        B.K = f->args;
        B.K.ustg = R.ws + R.off_stage + ((size_t)(n - s0) * 4 + (st - 1)) * z.stage_slot;
        B.K.use_dev_time = 0;
        B.K.t = th[n - s0] + (st == 1 ? 0.0 : (st == 4 ? dt : 0.5 * dt));
        B.K.stage = 0;
        if (mixed) {
          // the FP64 shadow: traces into the workspace, analytic velocity
          const char* U = static_cast<const char*>(B.K.ustg);
          B.K = shadow_args(f, R);
          B.K.ustg = const_cast<char*>(U);
          B.K.use_dev_time = 0;
          B.K.t = th[n - s0] + (st == 1 ? 0.0 : (st == 4 ? dt : 0.5 * dt));
          B.K.stage = 0;
          ks64.ka[0](B.K, s);
        } else {
          f->ks.ka[0](B.K, s);  // traces of this stage input
        }
        B.lamk = st == 4 ? Lp : Lk;
        B.lam_scale = st == 4 ? dt / 6.0 : 1.0;
        B.Y = Y;
        B.lamU = lamU;
        B.lamuo = lamuo;
        B.coefp = coefp;
        B.want_coef = M2 > 0;
        B.lv = lv;
        B.Lp = Lp;
        B.Lu = Lu;
        B.first = st == 4;
        switch (st) {
          case 4: B.Lk = Lk; B.c_lp = dt / 3.0; B.c_a = dt; break;
          case 3: B.Lk = Lk; B.c_lp = dt / 3.0; B.c_a = 0.5 * dt; break;
          case 2: B.Lk = Lk; B.c_lp = dt / 6.0; B.c_a = 0.5 * dt; break;
          default: B.Lk = nullptr; B.c_lp = 0.0; B.c_a = 0.0;
        }
        as.a(B, s);
        as.b(B, s);
        if (M2) {
          const double T = f->prm.vel.T;
          const double gt = T > 0.0 ? std::cos(M_PI * B.K.t / T) : 1.0;  // time factor of this stage
          k_coef_acc<<<R.adj_blocks, 256, 0, s>>>(lv, cs, npts, f->args.cd.vel, gt, coefp);
        }
        // adj_c reads Lk (through lamk of the next stage) only after this stage
        // is complete; writing Lk here is safe because stage st consumed it in adj_a/adj_b
        as.c(B, s);
      }
      std::swap(Lp, Lu);
    }
  }
  CK(cudaGetLastError());
  k_unpack_lam<<<grid, 256, 0, s>>>(Lp, dJ_du0, E, NU);
  if (R.precond) {
    // reverse sweep through the pseudo iterations of the t = 0
    // preconditioning: phi is not changed by them (its adjoint, kept in
    // dJ_du0, is carried with zero weight), psi's is propagated to psi(0) =
    // phi0 - 1/2, and the dependence of the source on psi0 = phi0 - 1/2 is
    // accumulated
    double* lpsi0 = reinterpret_cast<double*>(R.ws + R.off_lpsi0);
    k_zero_phi<<<grid, 256, 0, s>>>(Lp, E, NU);
    CK(cudaMemsetAsync(lpsi0, 0, (size_t)E * NU * 8, s));
    const double dtau = f->prm.pseudo_dtau;
    for (int k = R.n_pseudo - 1; k >= 0; --k) {
      for (int st = 4; st >= 1; --st) {
        AdjArgs B;
        std::memset(&B, 0, sizeof(B));
        B.K = f->args;
        B.K.ustg = R.ws + R.off_pstage + ((size_t)k * 4 + (st - 1)) * z.stage_slot;
        B.K.use_dev_time = 0;
        B.K.t = 0.0;
        B.K.stage = 0;
        if (mixed) {
          const char* U = static_cast<const char*>(B.K.ustg);
          B.K = shadow_args(f, R);
          B.K.ustg = const_cast<char*>(U);
          B.K.use_dev_time = 0;
          B.K.t = 0.0;
          B.K.stage = 0;
          ks64.ka[0](B.K, s);
        } else {
          f->ks.ka[0](B.K, s);
        }
        B.lamk = st == 4 ? Lp : Lk;
        B.lam_scale = st == 4 ? dtau / 6.0 : 1.0;
        B.Y = Y;
        B.lamU = lamU;
        B.lamuo = lamuo;
        B.Lp = Lp;
        B.Lu = Lu;
        B.first = st == 4;
        B.lam_psi0 = lpsi0;
        switch (st) {
          case 4: B.Lk = Lk; B.c_lp = dtau / 3.0; B.c_a = dtau; break;
          case 3: B.Lk = Lk; B.c_lp = dtau / 3.0; B.c_a = 0.5 * dtau; break;
          case 2: B.Lk = Lk; B.c_lp = dtau / 6.0; B.c_a = 0.5 * dtau; break;
          default: B.Lk = nullptr; B.c_lp = 0.0; B.c_a = 0.0;
        }
        as.a(B, s);
        as.b1(B, s);
        as.c(B, s);
      }
      std::swap(Lp, Lu);
    }
    CK(cudaGetLastError());
    k_precond_out<<<grid, 256, 0, s>>>(dJ_du0, Lp, lpsi0, E, NU);
  }
  if (M2 && dJ_dcoef) k_coef_reduce<<<1, 64, 0, s>>>(coefp, R.adj_blocks, M2, dJ_dcoef);
  // leave the field at the end of the recorded window
  char* last = R.ws + R.off_ckpt + (size_t)z.n_ckpt * z.ckpt_slot;
  CK(cudaMemcpyAsync(f->args.u, last, ubytes, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(f->args.dstate + DS_TIME, last + ubytes, 8, cudaMemcpyDeviceToDevice, s));
  const int rc = field_stage_and_traces(f, s);
  if (rc) return rc;
  f->nstep = nstep_save;
  CK(cudaStreamSynchronize(s));
  CK(cudaGetLastError());
  return FR_OK;
}
