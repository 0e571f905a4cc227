/*
 * fr_pcpf.h -- C ABI of the GB300 FR-PCPF library (libfrpcpf.so).
 *
 * The library advances the preconditioned conservative phase field of
 * arXiv 2006.10967 with explicit high-order Flux Reconstruction (FR) on
 * quadrilateral, triangular and hexahedral meshes:
 *
 *   phi_t + div(phi u) = div( max(gamma,|u|) (eps grad phi
 *                              - gamma phi(1-phi) grad psi/|grad psi|) )
 *                        (Section 2, Eq. altconservativephasefieldeq, with the
 *                         normal from psi as in Section 2's preconditioned form)
 *   psi_t + div(psi u) = 0                                   (Section 2)
 *   every N steps: psi0 = phi - 1/2, then pseudo-time iterations of
 *   psi_tau = div(nu_s grad psi) + sgn(psi0)(1 - |grad psi|)
 *                        (Section 2 Eq. lsequation; Section 3.2
 *                         Eqs. peudoSystem1, resolutionIndicator, nu_s,
 *                         pseudotimesystem and the L2 stop rule)
 *
 * Spatial discretisation: FR Steps 1-6 of Section 3.1 (Eqs. extrapolateSoln,
 * continuousGrad, extrapolateGrad, normalTransFlux, commonFlux, inviscidFlux,
 * viscousFlux, continuousDivFlux), copy ghost states on walls (Section 3.3);
 * time: the 4-stage Runge-Kutta march of Section 3.1 (classical RK4).
 *
 * Conventions
 *  - All functions return an int status: FR_OK (0) or a negative FR_E* code.
 *    No exception or longjmp crosses this boundary.  fr_strerror() names codes.
 *  - "host" pointers are CPU memory, "device" pointers are CUDA device memory
 *    of the current device.  Host inputs are copied before the call returns;
 *    the caller keeps ownership of every pointer it passes.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it asynchronously unless stated otherwise.
 *  - The library never allocates device memory.  The caller allocates one
 *    workspace of fr_field_workspace_bytes() bytes (256-byte aligned) and
 *    passes it to fr_field_init(); it must outlive the field.
 *  - Solution-point data are laid out element-major: value (e, i) at index
 *    e * Nu + i, where i orders tensor points xi-fastest (then eta, zeta) on
 *    quadrilaterals/hexahedra and lattice points (i fastest, then j) on
 *    triangles; fr_mesh_solution_points() returns the coordinates.
 *  - Vertex orders: quad counter-clockwise; tri counter-clockwise; hex the
 *    quad order at zeta = -1 then at zeta = +1.
 */
#ifndef FR_PCPF_H
#define FR_PCPF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define FR_OK 0
#define FR_EINVAL (-1)      /* invalid argument, mesh or parameter */
#define FR_ENOMEM (-2)      /* host allocation failed or workspace too small */
#define FR_ECUDA (-3)       /* a CUDA runtime call failed */
#define FR_ENONFINITE (-4)  /* a non-finite value appeared in the state */
#define FR_ETIMEOUT (-5)    /* a bounded device wait gave up */
#define FR_EUNSUPPORTED (-6) /* element type / order / mode not built */
#define FR_EBOUNDS (-7)     /* a partner index read from the connectivity was out of
                               range (reported only by the bounds-checked build,
                               libfrpcpf_checked.so, whose kernels check every such
                               index before use and skip the access) */

/* ---- element types, precisions, velocity and IC kinds ---------------- */
#define FR_QUAD 0
#define FR_TRI 1
#define FR_HEX 2

#define FR_FP64 0  /* every array and operation in double precision */
#define FR_MIXED 1 /* float stage values/fluxes/traces; double solution,
                      RK accumulator, psi0 and mass integral */

#define FR_VEL_UNIFORM 0     /* u = a g(t) */
#define FR_VEL_RIDER_KOTHE 1 /* Section 4.2 field times g(t) */
#define FR_VEL_LEVEQUE 2     /* Section 4.3 field times g(t) */
#define FR_VEL_STREAM 3      /* u = dPsi/dy, v = -dPsi/dx,
                                Psi = g(t) sum_m A_m sin(2 pi k_m.x) + B_m cos(2 pi k_m.x) */
#define FR_VEL_ROTATION 4    /* solid-body rotation about (a[0], a[1]): (a[1] - y, x - a[0]),
                                Section 4.1 (Zalesak: centre (0.5, 0.5); Rudman: (2, 2)) */
#define FR_MAX_MODES 32

#define FR_IC_CIRCLE 0 /* phi = (1 + tanh(beta (r - |x - c|)))/2, Eqs. initialCond, discEq */
#define FR_IC_ARRAY 1  /* phi0 given at the solution points (host, E*Nu) */

typedef struct fr_mesh fr_mesh;   /* opaque, host side */
typedef struct fr_field fr_field; /* opaque, host handle to device state */

/* Mesh description (Section 3.1: elements, mapping, coinciding flux points). */
typedef struct fr_mesh_desc {
  int32_t dim;           /* 2 or 3 */
  int32_t etype;         /* FR_QUAD, FR_TRI (dim 2) or FR_HEX (dim 3) */
  int32_t order;         /* p: quad 1..6, tri 1..5, hex 1..5 */
  int32_t reserved;
  int64_t n_nodes;
  const double* nodes;   /* host, n_nodes * dim, node-major */
  int64_t n_elems;
  const int64_t* conn;   /* host, n_elems * nverts (4, 3 or 8) */
  int32_t periodic[3];   /* axis a periodic with period[a] */
  double period[3];
} fr_mesh_desc;

typedef struct fr_mesh_info {
  int32_t dim, etype, order, nu, nf, n_faces_per_elem;
  int64_t n_elems;
  int64_t n_dof;         /* n_elems * nu */
  int64_t n_boundary_fpts;
  double h;              /* average element size (quad/hex (|Omega|/E)^(1/d); tri sqrt(2|Omega|/E)) */
  double volume;         /* |Omega| */
} fr_mesh_info;

typedef struct fr_velocity {
  int32_t kind;          /* FR_VEL_* */
  int32_t n_modes;       /* FR_VEL_STREAM: 1..FR_MAX_MODES */
  double T;              /* g(t) = cos(pi t / T) if T > 0, else 1 */
  double a[3];           /* FR_VEL_UNIFORM: the velocity at g = 1; FR_VEL_ROTATION: the centre */
  const double* kx;      /* host, n_modes each (FR_VEL_STREAM), copied */
  const double* ky;
  const double* A;
  const double* B;
} fr_velocity;

typedef struct fr_params {
  double gamma;          /* 0.09 in the paper */
  double eps;            /* 0.06 h/p in the paper */
  double tau;            /* LDG penalty on phi (total flux out of L gets +tau(u_L-u_R)) */
  double tau_psi;        /* penalty on psi's advection flux (0: central) */
  double tau_pseudo;     /* LDG penalty in the preconditioning equation */
  double dt;             /* physical time step */
  int32_t n_precond;     /* precondition every n_precond steps (paper: 1000) */
  int32_t pseudo_kmax;   /* maximum pseudo iterations (paper: up to 20) */
  double pseudo_dtau;    /* pseudo time step */
  double pseudo_tol;     /* stop when RMS((psi^k - psi^{k-1})/dtau) <= tol (paper: 1/2) */
  int32_t pseudo_fixed;  /* 1: always run pseudo_kmax iterations */
  int32_t precision;     /* FR_FP64 or FR_MIXED */
  double s0, kappa, nu_max; /* Eq. nu_s */
  double delta;          /* guard: |grad psi| -> max(|grad psi|, delta) */
  fr_velocity vel;
  int32_t vel_cache;     /* 1: store the time-independent factor v(x) of u(x,t) = g(t) v(x)
                            at every solution and flux point at init (evaluated in FP64;
                            dim x (nu+nf) values per element in the stage precision) instead
                            of evaluating v(x) every stage; 0: evaluate in the kernels */
  int32_t normal;        /* interface normal of the sharpening term: FR_NORMAL_PSI (the
                            preconditioned method, n = grad psi/|grad psi|, Section 2) or
                            FR_NORMAL_PHI (the unpreconditioned conservative phase field,
                            Eq. altconservativephasefieldeq with n = grad phi/|grad phi|;
                            fr_step and set-up then never reset or precondition psi, which
                            is still advected but feeds nothing).  Other values: FR_EINVAL */
  int32_t wall;          /* wall faces of the physical system: FR_WALL_COPY (Section 3.3:
                            ghost states copy the interior, so the diffusive and sharpening
                            fluxes of the interior pass through the wall) or FR_WALL_NOFLUX
                            (an option of this library, not the paper's: the common normal
                            flux of both fields is zero at wall flux points, so that mass is
                            conserved on walled domains as on periodic ones; the
                            preconditioning keeps the copy ghost).  FR_WALL_NOFLUX has no
                            adjoint (fr_adjoint_record: FR_EUNSUPPORTED).  Other values:
                            FR_EINVAL */
  int32_t variant;       /* implementation of the residual and update kernels, all giving the
                            same result to round-off: 0 the default; fr_kernel_variants gives
                            the count for a mesh and precision (FR_MIXED: triangles 0 scalar
                            dot products, 1 the operator applies on tensor cores, mma.sync
                            m16n8k8 in three-term TF32 with FP32 accumulation; quads and hexes
                            the element tiles of the physical-step residual and update kernels:
                            0 default/default, 1 half/half, 2 default/half, 3 half/default).
                            An autotuner picks among them by measurement.  Out of range:
                            FR_EUNSUPPORTED from fr_field_init, negative: FR_EINVAL */
} fr_params;

enum { FR_NORMAL_PSI = 0, FR_NORMAL_PHI = 1 };
enum { FR_WALL_COPY = 0, FR_WALL_NOFLUX = 1 };

typedef struct fr_ic {
  int32_t kind;          /* FR_IC_CIRCLE or FR_IC_ARRAY */
  int32_t precondition;  /* 1: reset psi = phi - 1/2 and precondition (Section 2) */
  double centre[3];
  double radius;
  double beta;           /* sharpness; the paper uses 3p/(4h) */
  const double* phi0;    /* FR_IC_ARRAY: host, n_dof */
} fr_ic;

/* One instance of a batch (fr_field_init_batch): elements
 * [elem_begin, elem_end) of the union mesh with their own time step,
 * interface width eps, maximum artificial viscosity nu_max, pseudo time step,
 * velocity field and initial circle. */
typedef struct fr_instance {
  int64_t elem_begin, elem_end;
  double dt, eps, nu_max, pseudo_dtau;
  fr_velocity vel;       /* vel.T must equal the batch's params->vel.T */
  fr_ic ic;              /* FR_IC_CIRCLE; ic.precondition is ignored */
} fr_instance;

typedef struct fr_stats {
  int64_t n_steps;       /* physical steps taken since init */
  double t;              /* physical time */
  int32_t last_pseudo_iters;
  int32_t status;        /* sticky device status: FR_OK, FR_ENONFINITE, ... */
  double last_pseudo_rms;
  int64_t n_preconditions;
} fr_stats;

/* ---- mesh ------------------------------------------------------------ */

/* Build the host mesh: reference operators, element geometry, face pairing
 * (faces matched by vertex positions modulo the periods; flux points by
 * physical position).  The L side of an interior face is the lower element
 * number.  Unmatched faces are walls (copy ghost states, Section 3.3).
 * Errors: FR_EINVAL (bad dim/type/order/index, face shared by > 2 elements,
 * non-coinciding flux points, det J <= 0), FR_ENOMEM, FR_EUNSUPPORTED (order
 * not built, or n_elems * Nf >= 2^30: the packed partner index of a flux
 * point, 2 (e Nf + k) + L, is an int32; checked before the arrays are read). */
int fr_mesh_create(const fr_mesh_desc* desc, fr_mesh** out);
int fr_mesh_info_get(const fr_mesh* mesh, fr_mesh_info* info);
/* Physical solution-point coordinates, host out[n_dof * dim] (point-major). */
int fr_mesh_solution_points(const fr_mesh* mesh, double* out);
/* Quadrature weights w_i det J_ei, host out[n_dof]: the exact integral of the
 * interpolant (Section 4 error measures). */
int fr_mesh_quadrature(const fr_mesh* mesh, double* out);
void fr_mesh_destroy(fr_mesh* mesh);

/* Union of n meshes of the same element type and order (their elements in
 * order, each keeping its own faces and periodicity): the mesh of a batch of
 * independent instances.  Inputs are not modified. */
int fr_mesh_concat(const fr_mesh* const* meshes, int n, fr_mesh** out);

/* ---- field ----------------------------------------------------------- */

/* Bytes of device workspace fr_field_init needs for this mesh and params. */
int fr_field_workspace_bytes(const fr_mesh* mesh, const fr_params* prm, size_t* bytes);

/* Create a field on `workspace` (device, >= fr_field_workspace_bytes, 256-byte
 * aligned), set phi from `ic`, psi = phi - 1/2, and (if ic->precondition)
 * run the preconditioning of Section 2 at t = 0.  Synchronises `stream`.
 * Errors: FR_EINVAL, FR_ENOMEM (workspace too small), FR_ENONFINITE (IC not
 * finite), FR_EUNSUPPORTED, FR_ECUDA. */
int fr_field_init(const fr_mesh* mesh, const fr_params* prm, const fr_ic* ic,
                  void* workspace, size_t workspace_bytes, void* stream, fr_field** out);

/* A field over a batch of independent instances sharing one union mesh
 * (fr_mesh_concat of quad or hex meshes of one order): each instance marches
 * with its own dt, eps, nu_max, pseudo_dtau and velocity; gamma, tau, the
 * preconditioning schedule, the sensor ramp, the precision and the velocity
 * period come from `params`.  Needs params->vel_cache = 1 (the velocities are
 * stored per point).  The instances step together: fr_step(n) advances every
 * instance n of its own steps.  Preconditioning at t = 0 when `precondition`.
 * Errors as fr_field_init; FR_EUNSUPPORTED for triangles. */
int fr_field_init_batch(const fr_mesh* mesh, const fr_params* params, int n_instances,
                        const fr_instance* instances, int precondition, void* workspace,
                        size_t workspace_bytes, void* stream, fr_field** out);

/* Advance n_steps physical RK4 steps on `stream` (asynchronous).  Before step
 * n (n > 0, n % n_precond == 0) psi is reset to phi - 1/2 and preconditioned.
 * Returns the sticky status of earlier work (FR_ENONFINITE once a non-finite
 * value was seen); call fr_sync for the status of this call. */
int fr_step(fr_field* field, int n_steps, void* stream);

/* Reset psi0 = phi - 1/2 and run the pseudo-time iterations now (asynchronous). */
int fr_precondition(fr_field* field, void* stream);

/* Synchronise `stream`, read the device status word; returns it. */
int fr_sync(fr_field* field, void* stream);
int fr_stats_get(fr_field* field, void* stream, fr_stats* out);

/* int phi dOmega (which = 0) or int psi dOmega (which = 1): sum over elements
 * and points of w_i det J_i u_i with a compensated (Neumaier) FP64 reduction
 * in a fixed order (deterministic).  Synchronous: *out_host is valid on return. */
int fr_mass_integral(fr_field* field, int which, double* out_host, void* stream);

/* Allocation-free weighted integral.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc -- code running
 * inside another framework's memory pool (a cudaMalloc would bypass its
 * accounting and can fragment its arena), latency-critical loops that cannot
 * afford the implicit device synchronisation of cudaMalloc/cudaFree, and
 * callers that hold their data on the device without an fr_field workspace.
 *
 * Computes sum_i w[i] * u[i] over n doubles (dev_u, dev_w: device arrays,
 * caller-owned) with the same Neumaier-compensated FP64 method as
 * fr_mass_integral, in its own fixed order (contiguous blocks of 2048 values,
 * then the block partials in index order), so the result is deterministic
 * for a given n and agrees with fr_mass_integral to about 1e-13 relative
 * (the two summation orders differ).  The result is written to *out_host:
 * the call waits for the stream (cudaStreamSynchronize) before returning,
 * so it must not be called while that stream is being captured into a graph.
 * Pass u = one field from fr_field_get_device and w = fr_mesh_quadrature
 * copied to the device to compare with fr_mass_integral.
 *
 * Scratch: a static device array of FR_NOALLOC_MAX_BLOCKS (sum, compensation)
 * pairs plus two words (~256 KB), held by every GPU that loads the library
 * until the process exits.  n > FR_NOALLOC_MAX_VALUES returns FR_EINVAL.
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make that first call
 * before any stream capture.  All calls share the one array and each call
 * resets its counter before use, so calls that overlap on the GPU (other
 * streams, other host threads) race and must be serialised by the caller.
 * Allocates nothing: no cudaMalloc, cudaFree or allocating library call. */
#define FR_NOALLOC_MAX_BLOCKS 16384
#define FR_NOALLOC_MAX_VALUES ((int64_t)FR_NOALLOC_MAX_BLOCKS * 256 * 8)
int fr_mass_integral_noalloc(const double* dev_u, const double* dev_w, int64_t n, double* out_host,
                             void* stream);

/* Copy a field to/from host memory (synchronous): which = 0 phi, 1 psi,
 * 2 psi0; n_dof doubles.  fr_field_set also refreshes the stage copies and
 * flux-point traces. */
int fr_field_get(fr_field* field, int which, double* host, void* stream);
int fr_field_set(fr_field* field, int which, const double* host, void* stream);
/* Device-pointer variants (asynchronous on `stream`), n_dof doubles. */
int fr_field_get_device(fr_field* field, int which, double* dev, void* stream);
int fr_field_set_device(fr_field* field, int which, const double* dev, void* stream);

/* ---- groups ----------------------------------------------------------
 * A group steps several fields together with one launch of the residual
 * kernel and one of the update kernel per RK stage: block b of a launch
 * belongs to the field whose range of blocks holds b (a work list over the
 * fields' element tiles), and each field keeps its own state, time and
 * per-element parameters.  Built for the batched ensemble (Section 4's
 * workloads in an uneven ensemble): quadrilateral FR_MIXED fields of
 * distinct orders 2..5, with equal n_precond and step counts.  The physical
 * steps of all fields run as one launch sequence (captured in CUDA graphs);
 * a preconditioning due before a step runs per field (fr_precondition).
 * The fields must outlive the group and must not be stepped on their own
 * while it is used.  Errors: FR_EINVAL (null, n outside 1..4),
 * FR_EUNSUPPORTED (a field outside that set, two fields of one order,
 * differing n_precond or step counts), FR_ENOMEM, FR_ECUDA. */
typedef struct fr_group fr_group;
int fr_group_create(fr_field* const* fields, int n, fr_group** out);
/* n_steps RK4 steps of every field of the group, asynchronous on `stream`. */
int fr_group_step(fr_group* group, int n_steps, void* stream);
void fr_group_destroy(fr_group* group);

/* ---- element-partitioned runs (one rank per GPU) ------------------------
 * A rank holds the elements it owns plus the ghost elements within two
 * face-neighbour layers of them, all in one local mesh.  The residual of an
 * owned element (Section 3.1, Steps 1-6) reads its neighbours' traces
 * (Step 2) and, on faces where a neighbour is the L side, that neighbour's
 * corrected gradient (Step 5), which reads the neighbour's neighbours; so
 * with the ghosts' stage values taken from their owners before every RK
 * stage, the owned elements march exactly as in the whole mesh.  A rank
 * steps with fr_stage (one stage at a time) and, between stages, gathers the
 * stage values its peers need (fr_halo_pack), exchanges them (the caller's
 * transport: NCCL, or device copies), scatters the received ones into its
 * ghosts (fr_halo_unpack) and recomputes the flux-point traces
 * (fr_traces).  The ghosts' own updates are discarded by the next exchange.
 * The preconditioning runs the same way with fr_pseudo_begin and
 * fr_pseudo_stage in place of fr_stage (fixed iteration count only).
 *
 * fr_stage: stage s (1..4) of the physical RK4 step on `stream`, the
 * residual and update kernels of that stage (asynchronous; no CUDA graph);
 * stage 4 completes the step (the step count and time advance).  Errors:
 * FR_EINVAL (null, s outside 1..4). */
int fr_stage(fr_field* field, int stage, void* stream);
/* Bytes of one element's stage values (2 fields x nu values in the field's
 * bulk precision: 8-byte doubles for FR_FP64, 4-byte floats for FR_MIXED). */
int fr_halo_row_bytes(const fr_field* field, size_t* bytes);
/* Gather (pack) the stage values of the n elements listed in elems_dev
 * (device, int64 local element indices) into buf_dev (device, n rows of
 * fr_halo_row_bytes, in list order), or scatter (unpack) n rows of buf_dev
 * into the listed elements.  Asynchronous on `stream`.  Every index is
 * checked on the device: an index outside [0, E) is skipped and records
 * FR_EINVAL in the status word (fr_sync reports it).  Errors: FR_EINVAL
 * (null pointers with n > 0, n < 0), FR_ECUDA. */
int fr_halo_pack(fr_field* field, const int64_t* elems_dev, int64_t n, void* buf_dev, void* stream);
int fr_halo_unpack(fr_field* field, const int64_t* elems_dev, int64_t n, const void* buf_dev, void* stream);
/* Recompute every element's flux-point traces from its stage values (Step 1,
 * Eq. extrapolateSoln) after fr_halo_unpack.  Asynchronous. */
int fr_traces(fr_field* field, void* stream);
/* The preconditioning of an element-partitioned run, one pseudo stage at a
 * time (Section 2, Eq. lsequation and the reset psi_0 = phi - 1/2; Section
 * 3.2, Eq. pseudotimesystem marched by RK4 in pseudo time).  fr_pseudo_begin
 * resets psi_0 and psi from phi on every local element and computes psi's
 * traces; fr_pseudo_stage(s) runs stage s (1..4) of one pseudo-time
 * iteration with the pseudo time step params.pseudo_dtau.  A rank calls
 * fr_pseudo_begin, exchanges its ghosts (fr_halo_pack / fr_halo_unpack /
 * fr_traces, as after fr_stage), then for each of params.pseudo_kmax
 * iterations makes the four fr_pseudo_stage calls, each followed by the
 * same exchange; the owned elements then hold what fr_precondition gives
 * on the whole mesh.  Only
 * fields with params.pseudo_fixed = 1 (the stop rule's RMS over the local
 * points would count the ghosts) and the preconditioned normal
 * (FR_NORMAL_PSI): FR_EUNSUPPORTED otherwise.  Asynchronous on `stream`; no
 * CUDA graph.  Errors: FR_EINVAL (null field, stage outside 1..4),
 * FR_EUNSUPPORTED, FR_ECUDA. */
int fr_pseudo_begin(fr_field* field, void* stream);
int fr_pseudo_stage(fr_field* field, int stage, void* stream);

/* Number of kernel variants (fr_params.variant) built for the mesh's element
 * type and order in `precision` (FR_FP64 or FR_MIXED): *count >= 1. */
int fr_kernel_variants(const fr_mesh* mesh, int precision, int32_t* count);

/* Measurement entry point: the element-local operator applies of Steps 1 and
 * 3 on hexahedra of order 3 (Section 3.1, Eq. extrapolateSoln: the flux-point
 * traces u^f = L u; Eq. continuousGrad: the reference derivatives D_a u,
 * without the correction terms) in one of two forms, so that they can be
 * timed against each other:
 *   form 0: the 1D operators along solution-point lines (sum factorisation,
 *           the form of the residual kernel), FP32 FMAs;
 *   form 1: the dense 288 x 64 operator [L; D_0; D_1; D_2] on the tensor
 *           cores (mma.sync m16n8k8, three-term TF32, FP32 accumulation).
 * u_dev: device, n_elems x 2 x 64 floats (element, field, solution point;
 * the stage-value layout), 16-byte aligned.  out_dev: device, out_len
 * floats.  reduce == 0: n_elems x 2 x 288 values; per (element, field) the
 * 96 traces (face 2a + sd, face point l: line l along axis a, the other two
 * point indices with the lower axis fastest), then the derivatives along
 * axes 0, 1, 2 at the 64 points.  reduce != 0: n_elems x 2 values, the sum of
 * each (element, field)'s 288 values (for timing without the output
 * traffic).  Asynchronous on `stream`.  Errors: FR_EUNSUPPORTED (order != 3),
 * FR_EINVAL (form not 0 or 1, negative n_elems, null or misaligned pointers,
 * out_len too small), FR_ECUDA. */
int fr_probe_hex_apply(int order, int form, int reduce, const float* u_dev, int64_t n_elems,
                       float* out_dev, int64_t out_len, void* stream);

/* Evaluate the semi-discrete right-hand side du/dt = -J^{-1} div~ f~ (Step 6)
 * of the physical system at the current state and time t into dev_out
 * (device, 2 * n_dof doubles: phi rates then psi rates).  Does not change the
 * state.  Asynchronous. */
int fr_rhs(fr_field* field, double t, double* dev_out, void* stream);
/* Same for the preconditioning system (Eq. pseudotimesystem), psi rates into
 * dev_out (n_dof doubles), with the stored psi0. */
int fr_rhs_pseudo(fr_field* field, double* dev_out, void* stream);

/* ---- discrete adjoint ---------------------------------------------------
 * The paper has no adjoint; these calls give the exact gradient of the FR
 * march's discrete map for a loss of the final state, with respect to the
 * initial fields and the stream-function coefficients (FR_VEL_STREAM).
 * Built for quadrilaterals (p <= 6), hexahedra (p <= 3) and triangles
 * (p <= 5) in both precisions.  On an FR_MIXED field the
 * recorded march is the field's own FP32 one (its float-float states are the
 * checkpoints); the sweep recomputes each segment in FP64 from its widened
 * checkpoint on FP64 shadow arrays in the workspace (a preconditioning in the
 * window likewise from phi0) and applies the FP64 vector-Jacobian products
 * along that recomputation (velocity evaluated analytically): the FP64
 * scheme's gradient along trajectories restarted every ckpt_every steps from
 * the FP32 march.  (Along the FP32 stage inputs themselves the linearisation
 * is ill-conditioned: psi rounded to float has flat spots where phi is small,
 * where the normal's derivative is 1/delta.)  The recorded window must not
 * contain a preconditioning step (n > 0, n % n_precond == 0).
 *
 * flags: 0, or FR_ADJ_PRECONDITION: the window starts with the
 *   preconditioning of Section 2 from the current phi (psi0 = psi = phi -
 *   1/2, then pseudo_kmax pseudo-time RK4 iterations of Eq. pseudotimesystem;
 *   needs params.pseudo_fixed = 1), and dJ_du0 of fr_adjoint_step is then
 *   dJ/dphi0 along both paths, phi0 itself and psi = P(phi0 - 1/2) with the
 *   source's psi0 = phi0 - 1/2 (its psi half is zero: psi is no input).
 * fr_adjoint_workspace_bytes: device bytes for a window of n_steps with a
 *   checkpoint every ckpt_every steps ((n_steps/ckpt_every + 1) solution
 *   copies + 4 * ckpt_every stage inputs + adjoint work arrays; with
 *   FR_ADJ_PRECONDITION also 4 * pseudo_kmax pseudo stage inputs).
 * fr_adjoint_record: advance n_steps from the current state (as fr_step),
 *   keeping checkpoints in `workspace` (device, caller-owned, 256-byte
 *   aligned, >= the bytes above; it must live until fr_adjoint_step returns).
 *   FR_EUNSUPPORTED for a field whose normal is FR_NORMAL_PHI (the adjoint
 *   covers the preconditioned method), for no-flux walls, for batch fields
 *   (fr_field_init_batch: per-instance time steps), and for FR_ADJ_PRECONDITION without
 *   pseudo_fixed (the stop rule's iteration count is not differentiated).
 * fr_adjoint_step: given dJ/dphi(T) (device, n_dof) and optionally dJ/dpsi(T)
 *   (device, n_dof, or NULL for zero), write dJ/du(t0) to dJ_du0 (device,
 *   2 * n_dof: phi then psi) and, for a stream-function velocity,
 *   dJ/d(A_1..A_M, B_1..B_M) to dJ_dcoef (device, 2M, or NULL).  Recomputes
 *   the forward stages segment by segment from the checkpoints; on return the
 *   field is back at the end of the window.  Synchronises `stream`. */
#define FR_ADJ_PRECONDITION 1
int fr_adjoint_workspace_bytes(fr_field* field, int n_steps, int ckpt_every, int flags, size_t* bytes);
int fr_adjoint_record(fr_field* field, int n_steps, int ckpt_every, int flags, void* workspace,
                      size_t workspace_bytes, void* stream);
int fr_adjoint_step(fr_field* field, const double* dJ_dphiT, const double* dJ_dpsiT, double* dJ_du0,
                    double* dJ_dcoef, void* stream);

/* Per-kernel timing (not part of the method): with enable != 0 every FR
 * kernel launch of fr_step / fr_precondition is bracketed by CUDA events on
 * its stream.  fr_profile_read synchronises `stream` and returns, for the
 * four kernel classes {residual+flux (physical), lift+RK+traces (physical),
 * residual+flux (preconditioning), lift+RK+traces (preconditioning)}, the
 * summed device milliseconds and the launch counts since the last read
 * (host arrays of 4). */
int fr_profile(fr_field* field, int enable);
int fr_profile_read(fr_field* field, void* stream, double* total_ms, int64_t* launches);

/* Steady-state duration of one kernel class (not part of the method): n
 * back-to-back launches of the class on the field's current state, replayed
 * as one CUDA graph on `stream` after one untimed replay, bracketed by CUDA
 * events; *ms_per_launch receives the mean milliseconds per launch.  kernel 0
 * is the physical residual + common flux kernel (Steps 1-6 of Section 3.1) at
 * RK stage 1.  The state is unchanged; the partial residual and common-flux
 * scratch is overwritten (every step rewrites it).  FR_EINVAL for another
 * class, n < 1 or a NULL pointer.  Synchronises `stream`. */
int fr_profile_kernel(fr_field* field, int kernel, int n, void* stream, double* ms_per_launch);

void fr_field_destroy(fr_field* field);

const char* fr_strerror(int code);
int fr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FR_PCPF_H */
