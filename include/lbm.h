/*
 * lbm.h -- C ABI of the B300 (sm_103a) total-Lagrangian vectorial lattice
 * Boltzmann library for finite-strain hyperelasticity on embedded curved
 * domains (arXiv 2606.20646).
 *
 * The calls follow the paper's statement of the problem: a reference body
 * given by a level set (Sec. 3.1, Eq. level-set-domain) on a Cartesian
 * lattice, a hyperelastic material (Sec. 4.1, Eq. validation-nh-energy),
 * boundary data on Dirichlet and nominal-traction parts of the surface
 * (Sec. 2.1, Eqs. physical-dirichlet, vD-from-uD, nominal-traction-general),
 * initial fields (Eq. initial-data-general), and the one-step update of
 * Algorithm 1 (Sec. 3.6), returning the fields v, F and u.
 *
 * Conventions shared by every call
 *   - Lattice nodes are cell centred: X_i = origin + (i + 1/2) dx.
 *   - Box fields are structure-of-arrays planes of doubles, one plane per
 *     component, each plane nx*ny*nz values with x fastest (node index
 *     x + nx*(y + ny*z)); inactive nodes are written as 0 and ignored on input.
 *     v: D planes; F: D*D planes, F row-major (F_11, F_12, .., F_DD) as in
 *     Eq. (state-general-d); u: D planes; dU0: D*(D+D*D) planes, plane
 *     A*(D+D*D) + k holding d U0_k / d X_A.
 *   - Pointers to fields may be device pointers, or host pointers when the
 *     handle was created with host staging (lbm_options.host_staging = 1);
 *     the library tells them apart with cudaPointerGetAttributes.
 *   - All device work is enqueued on the CUDA stream given to lbm_create and
 *     is asynchronous unless stated otherwise.  Device-side failures (Newton
 *     non-convergence, J <= 0, non-finite values) are latched in a device
 *     status word and reported by lbm_sync.
 *   - The library never allocates device memory.  The caller allocates the
 *     geometry storage before lbm_create and the solver storage after it,
 *     keeps both alive until lbm_destroy, and frees them afterwards.  The
 *     handle itself owns only host memory.
 *   - Every int-returning call returns LBM_OK (0) or a negative lbm_error;
 *     lbm_error_string gives its text.  No call throws or aborts.
 */
#ifndef LBM_B300_H
#define LBM_B300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes (negative returns) -------------------------------------- */
enum lbm_error {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,      /* invalid argument or descriptor                           */
    LBM_ERR_DOMAIN = -2,   /* empty body, or the body extends past a non-periodic box face */
    LBM_ERR_CUDA = -3,     /* a CUDA runtime call failed                               */
    LBM_ERR_STORAGE = -4,  /* storage missing, too small or misaligned (256 B)         */
    LBM_ERR_STATE = -5,    /* call out of order (e.g. lbm_step before lbm_set_initial) */
    LBM_ERR_DEVICE = -6,   /* lbm_sync found a non-zero device status word             */
    LBM_ERR_CAPACITY = -7, /* a fixed capacity was exceeded (LSQ stencil, census box)  */
    LBM_ERR_UNSTABLE_C = -8 /* the lattice speed c fails the tangent wave-speed audit   */
};

/* ---- device status bits returned by lbm_sync ------------------------------ */
enum lbm_device_status {
    LBM_DEV_NONFINITE = 1, /* a recovered state component was not finite             */
    LBM_DEV_JACOBIAN = 2,  /* J = det F <= 0 at an active node (Eq. positive-jacobian) */
    LBM_DEV_NEWTON = 4,    /* traction inversion failed (Eqs. neumann-newton-2d/3d)   */
    LBM_DEV_LSQ = 8,       /* no least-squares fit at a Neumann link                   */
    LBM_DEV_CAPACITY = 16, /* LSQ stencil larger than LBM_LSQ_CAPACITY                */
    LBM_DEV_TIMEOUT = 128, /* a bounded wait for a TMA copy ran out; that step is invalid */
    LBM_DEV_BOUNDS = 256   /* bounds-checked build only: an index left its array (the access
                              was redirected to element 0); the results are invalid        */
};

/* FP64: populations and arithmetic in FP64.  FP32: both in FP32, populations stored shifted
 * (f - f^eq(0, I)).  BF16S: the FP32 form with the shifted populations stored as BF16 (rounded to
 * nearest even on store; every other array, the cut links' kept and reconstructed values and the
 * displacement accumulators keep their FP32 form); half the population bytes of FP32.  Not with
 * options.adjoint. */
enum lbm_precision { LBM_PREC_FP64 = 0, LBM_PREC_FP32 = 1, LBM_PREC_BF16S = 2 };

/* level-set primitives; local coordinates xi = rot^T (X - center), rot row-major 3x3
 *   SPHERE        phi = |X - center| - axes[0]                (circle in 2D)
 *   ELLIPSOID     phi = sum_a (xi_a / axes[a])^2 - 1          (ellipse in 2D)
 *   SUPERELLIPSE  phi = |xi_1/axes[0]|^p + |xi_2/axes[1]|^p - 1  (2D only)
 *   CYLINDER      phi = |(X_1, X_2) - (c_1, c_2)| - axes[0]   (axis X_3)
 *   HALFSPACE     phi = axes . (X - center), axes a unit outward normal
 *   SAMPLED       phi given at the lattice nodes (lbm_shape.phi: n_box doubles in box order, device
 *                 memory the caller keeps valid until lbm_destroy); between nodes the multilinear
 *                 interpolant (linear along every link, so eta is the root of a linear function),
 *                 constant beyond the outermost node of a non-periodic axis (a sampled body must
 *                 not reach such a face: the box-face rule refuses it), periodic on periodic axes;
 *                 N_b (Eq. level-set-normal) from the same interpolant of the nodes' central
 *                 differences (one-sided at non-periodic ends); center, axes, rot unused
 * complement != 0 negates phi.  The body is {X : max_s phi_s(X) <= 0}. */
enum lbm_shape_kind {
    LBM_SHAPE_SPHERE = 0,
    LBM_SHAPE_ELLIPSOID = 1,
    LBM_SHAPE_SUPERELLIPSE = 2,
    LBM_SHAPE_CYLINDER = 3,
    LBM_SHAPE_HALFSPACE = 4,
    LBM_SHAPE_SAMPLED = 5
};

enum lbm_bc_kind { LBM_BC_DIRICHLET = 0, LBM_BC_NEUMANN = 1 };

/* boundary profiles, s(t) the ramp:
 *   Dirichlet (prescribed displacement; the lattice imposes v_D = d u_D / dt):
 *     ZERO          u_D = 0
 *     AFFINE        u_D = s(t) A (X - center)
 *     RADIAL        u_D = amp s(t) (X - center)/|X - center|
 *     TWIST_STRETCH u_D = ((R(s(t) amp) - I) (X_1 - c_1, X_2 - c_2), s(t) vec[2])  (3D)
 *     CONST         u_D = s(t) vec  (a translation of the boundary part)
 *   Neumann (nominal traction T = P N):
 *     CONST         T = s(t) vec
 *     RADIAL        T = amp s(t) (X - center)/|X - center|                        */
enum lbm_profile {
    LBM_PROFILE_ZERO = 0,
    LBM_PROFILE_AFFINE = 1,
    LBM_PROFILE_RADIAL = 2,
    LBM_PROFILE_TWIST_STRETCH = 3,
    LBM_PROFILE_CONST = 4
};

/* ramps: ONE s=1; LINEAR t/T then 1; SIN2 sin^2(pi t/(2T)) then 1 (Eq. sine2-ramp);
 * COS (1 - cos(pi t/T))/2 then 1 (Eq. tube-cosine-ramp); TIME s = t */
enum lbm_ramp { LBM_RAMP_ONE = 0, LBM_RAMP_LINEAR = 1, LBM_RAMP_SIN2 = 2, LBM_RAMP_COS = 3, LBM_RAMP_TIME = 4 };

/* initialisation: EQUILIBRIUM f = f^eq(U0); CHARACTERISTIC adds the second-order
 * correction of Eqs. (init-general-d, Ut-general-init) */
enum lbm_init { LBM_INIT_EQUILIBRIUM = 0, LBM_INIT_CHARACTERISTIC = 1 };

#define LBM_MAX_SHAPES 1024
#define LBM_MAX_GROUPS 256
#define LBM_MAX_BCS 16
#define LBM_LSQ_CAPACITY 160 /* max active nodes within 3 dx of a boundary point */

typedef struct lbm_grid {
    int dim;         /* 2 (D2Q4x6) or 3 (D3Q6x12)                               */
    int n[3];        /* nodes per axis; n[2] ignored in 2D                      */
    int periodic[3]; /* non-zero: periodic axis (no cut links across it)        */
    int reserved;
    double dx;       /* lattice spacing                                          */
    double origin[3];
} lbm_grid;

typedef struct lbm_shape {
    int kind;        /* enum lbm_shape_kind                                     */
    int complement;  /* non-zero: use -phi                                      */
    int boundary_id; /* id carried by cut links whose X_b lies on this shape    */
    int reserved;
    double center[3];
    double axes[3];
    double rot[9];
    double p;        /* superellipse exponent                                   */
    const double *phi; /* SAMPLED: the node samples (device memory), else unused */
} lbm_shape;

typedef struct lbm_material {
    double mu;     /* shear modulus                  */
    double lambda; /* Lame's first parameter          */
} lbm_material;

/* A body of several disjoint specimens (no counterpart in the paper, which treats one body at a
 * time): each group is one specimen, phi_g = max over the group's shapes, and the domain is the
 * union, phi = min over the groups whose box [lo, hi] contains X (phi > 0 outside every box).  A
 * group's box must contain its body.  Each group carries its own material; cut links take the
 * shape (and so the boundary id) of the group that defines phi at X_b. */
typedef struct lbm_group {
    int first_shape;  /* the group's shapes are shapes[first_shape .. first_shape + nshapes) */
    int nshapes;
    double lo[3], hi[3];
    lbm_material material;
} lbm_group;

typedef struct lbm_levelset {
    int nshapes; /* 0: every box node active (periodic boxes) */
    const lbm_shape *shapes;
    int ngroups; /* 0: one body, phi = max over all shapes, the material passed to lbm_create */
    const lbm_group *groups;
} lbm_levelset;

typedef struct lbm_bc {
    int boundary_id;
    int kind;    /* enum lbm_bc_kind */
    int profile; /* enum lbm_profile */
    int ramp;    /* enum lbm_ramp    */
    double t_ramp;
    double center[3];
    double A[9]; /* row-major 3x3 */
    double vec[3];
    double amp;
} lbm_bc;

typedef struct lbm_options {
    int precision;    /* enum lbm_precision: population storage and arithmetic              */
    int proj_every;   /* compatibility projection cadence in steps (0: never)            */
    int proj_iters;   /* damped-Jacobi sweeps per projection solve                        */
    int host_staging; /* non-zero: reserve a staging area so field calls accept host memory */
    double c;         /* lattice speed dx/dt                                              */
    double omega;     /* BGK relaxation, 0 < omega <= 2                                   */
    double gamma;     /* velocity damping: B = (b - gamma v, 0)                           */
    double theta_F;   /* F repair weight, 0 < theta_F <= 1 (Eq. projection-F-repair-weight) */
    double proj_beta; /* Jacobi damping, 0 < beta <= 1                                    */
    double body_force[3];
    int adjoint;      /* non-zero: reserve a per-node shear-modulus field and the reverse-mode
                         buffers of lbm_adjoint_* (Dirichlet-only bodies)                    */
    int reserved;
    double c_audit;   /* wave-speed audit (Sec. 2, Eq. acoustic-tensor-general-d): lbm_create and
                         lbm_set_initial require c >= c_audit * c_T, c_T the largest tangent wave
                         speed sqrt(max_n eig Q(n; F)) of the reference state F = I of every material
                         and of the initial F0 at every active node (rho0 = 1).  0 selects 2.5 (the
                         margin every closure case of the library's tests needed at omega = 1.8; the
                         bulk lattice alone needs sqrt(D)); a negative value turns the audit off */
} lbm_options;

typedef struct lbm_info {
    long long n_box, n_active, n_cut, n_neumann, n_dirichlet, n_segments;
    long long step;          /* steps taken since lbm_set_initial */
    double t, dt;
    size_t geometry_bytes, storage_bytes;
    long long launches;      /* kernels launched by lbm_step since creation */
    long long lsq_entries;   /* total LSQ stencil entries over Neumann links */
} lbm_info;

typedef struct lbm_kernel_time {
    double stream_collide_ms; /* fused gather + closure + collision kernel       */
    double cutlink_ms;        /* per-link boundary source kernel                  */
    double projection_ms;     /* projection, repair and reset kernels             */
    long long stream_collide_launches, cutlink_launches, projection_launches;
    double jacobi_ms;         /* damped-Jacobi sweeps alone (part of projection_ms) */
    long long jacobi_launches; /* the sweeps jacobi_ms covers (two per launch with two-sweep launches) */
} lbm_kernel_time;

typedef struct lbm_handle lbm_handle;

/* Bytes of caller-provided device memory lbm_create needs for the geometry
 * pass (active mask, cut-link bits, link offsets, segment list).  Depends only
 * on the grid.  Returns LBM_ERR_ARG for an invalid grid. */
int lbm_geometry_bytes(const lbm_grid *grid, size_t *bytes);

/* Validates the descriptors, then runs the FP64 geometry pass on the GPU in
 * geometry_storage (>= lbm_geometry_bytes, 256-byte aligned): active nodes
 * phi(X) <= 0 (Eq. level-set-domain) and cut links (Sec. 3.1, the sets I and
 * C of Sec. 3.6).  Synchronises the stream once to read the counts.  The
 * descriptors are copied; the arrays they point to may be freed on return.
 * Errors: LBM_ERR_ARG (bad descriptor, omega outside (0,2], dx<=0, c<=0,
 * missing BC for a boundary id is reported later by lbm_bind_storage),
 * LBM_ERR_DOMAIN (no active node, or the body extends past a non-periodic box
 * face: a cut link leaving the box must cross the surface within one spacing),
 * LBM_ERR_STORAGE, LBM_ERR_CUDA. */
int lbm_create(const lbm_grid *grid, const lbm_levelset *levelset, const lbm_material *material,
               const lbm_bc *bcs, int nbc, const lbm_options *options, void *geometry_storage,
               size_t geometry_bytes, void *cuda_stream, lbm_handle **out);

/* Bytes of solver storage (populations x2, u*, u^n, cut-link records, LSQ
 * weights, projection scratch, optional host staging). */
int lbm_storage_bytes(const lbm_handle *h, size_t *bytes);

/* Binds the solver storage (>= lbm_storage_bytes, 256-byte aligned) and builds
 * the per-link geometry in FP64 on the GPU: eta by bisection of phi
 * (Eq. cut-link-point), boundary normal (Eq. level-set-normal), boundary id,
 * tangent frame and LSQ tangent-derivative weights (Eq. tangent-derivative-2d,
 * Eq. tangent-image-3d-lsq).  Errors: LBM_ERR_STORAGE, LBM_ERR_ARG (a boundary
 * id with no BC), LBM_ERR_CAPACITY, LBM_ERR_CUDA. */
int lbm_bind_storage(lbm_handle *h, void *storage, size_t bytes);

/* Initial state (Eq. initial-data-general): v0 (D planes), F0 (D*D planes),
 * u0 (D planes), all required; dU0 (D*(D+D*D) planes) optional.  mode
 * LBM_INIT_EQUILIBRIUM sets f = f^eq(U0); LBM_INIT_CHARACTERISTIC applies
 * Eq. (init-general-d) with d_t U0 from Eq. (Ut-general-init), using dU0 when
 * given and second-order central (one-sided at the body) differences
 * otherwise.  Sets u*^0 = u0 - dt/2 v0 and the step counter to 0. */
int lbm_set_initial(lbm_handle *h, int mode, const double *v0, const double *F0, const double *u0,
                    const double *dU0);

/* Advances nsteps steps of Algorithm 1 (collide, stream, cut-link closure,
 * and, when Neumann links exist, the compatibility projection every
 * proj_every steps).  Enqueued; returns after launching. */
int lbm_step(lbm_handle *h, int nsteps);

/* The same nsteps steps recorded as one CUDA graph (stream capture of the launches lbm_step
 * would enqueue) and launched once on the handle's stream; no counterpart in the paper.  The
 * launches are recorded on a non-blocking stream the library creates for the handle on first use
 * (the handle's stream may be the legacy default stream, which cannot be captured) and destroys
 * in lbm_destroy.  The graph's kernel parameters (times, buffers) belong to these steps, so it is
 * launched once and kept until the next lbm_step_graph call or lbm_destroy.  The handle's stream
 * must not be capturing and kernel timing must be off.  Errors: LBM_ERR_ARG, LBM_ERR_STATE (not
 * initialised, timing on, or the stream capturing), LBM_ERR_CUDA (stream creation, capture,
 * instantiation or launch failed). */
int lbm_step_graph(lbm_handle *h, int nsteps);

/* ---- tile shapes ---------------------------------------------------------------------------
 * No counterpart in the paper.  Every choice below computes the same values node for node (the
 * fields are bit-identical); only the launch shape differs.  0 selects the form's default. */
typedef struct lbm_tuning {
    int windows_per_warp; /* fused kernel (bulk-copy forms): 32-node windows one warp stages at
                             once, 1, 2 or 4 (default 1 for FP32, 2 for BF16S)                  */
    int jacobi_segments;  /* projection sweeps: 32-node segments per warp, 1, 2 or 4 (default 1) */
    int link_block;       /* link kernel: threads per block, 64, 128 or 256 (default 128)        */
    int jacobi_sweeps;    /* projection: sweeps per launch, 1 or 2.  2 is available for the FP32
                             forms of boxes with no periodic axis (tiles staged by bulk copies, two
                             sweeps per pass over memory) and is the default there in 2D; 1 is the
                             default in 3D and the only choice elsewhere                          */
    int candidates;       /* lbm_autotune: configurations it timed                              */
    double ms_per_step;   /* lbm_autotune: the chosen configuration's time per step             */
    double default_ms_per_step; /* lbm_autotune: the defaults' time per step                     */
} lbm_tuning;

/* Sets the tile shapes (the last three fields are ignored; 0 in a field selects its default).
 * The shapes change no value: two sweeps per launch are bit-identical to two single sweeps.
 * Errors: LBM_ERR_ARG (a value outside its list). */
int lbm_set_tuning(lbm_handle *h, const lbm_tuning *t);
int lbm_get_tuning(const lbm_handle *h, lbm_tuning *t);

/* Autotuner: from the current state, times `steps` steps (CUDA events on the handle's stream, one
 * untimed step first) for each candidate shape, coordinate by coordinate (windows per warp, then
 * Jacobi segments and sweeps per launch when the body has Neumann links, then the link block when
 * it has cut links),
 * restoring the state after each run from `scratch` (lbm_state_bytes bytes of device memory, 256-byte
 * aligned; the library allocates nothing), keeps the fastest shapes and reports them in *out (may
 * be NULL).  The state on return is the state on entry.  Synchronises.  steps should cover a
 * projection step when the body has one (steps >= proj_every).  Errors: LBM_ERR_ARG, LBM_ERR_STATE
 * (not initialised, timing on, or a reverse sweep in progress), LBM_ERR_CUDA, LBM_ERR_DEVICE (a run
 * latched a device status; the state is restored). */
int lbm_autotune(lbm_handle *h, int steps, void *scratch, lbm_tuning *out);

/* Bounded waits (no counterpart in the paper).  The bulk-copy kernels poll the barrier of their
 * copies at most 2^20 times before they latch LBM_DEV_TIMEOUT, wait once more with that limit for
 * every copy they issued, and return without writing (the step is then invalid).  This sets the
 * first wait's limit (in the two-sweep Jacobi kernel, every wait's, after which the whole block
 * stops): 0 makes those waits run out at once, which tests that path without a fault; a negative
 * value restores 2^20.  Takes effect at the next launch. */
int lbm_set_wait_limit(lbm_handle *h, int polls);

/* ---- parameters, saved states and reverse mode --------------------------------------------
 * No counterpart in the paper: gradients of a loss on the final displacement with respect to a
 * per-node shear modulus and the body force, by the discrete adjoint of the steps (reverse
 * sweep over saved states).  Bodies with Neumann links (whose steps contain the Newton
 * inversion and the projection) are not supported: lbm_adjoint_begin returns LBM_ERR_STATE.
 * The initial populations are an input of the sweep, not differentiated: the gradients are those
 * of the steps.  A start from rest with F = I (P(I) = 0) makes them independent of mu and b, so
 * the gradients are then complete; a start in motion or strained (equilibrium or characteristic
 * populations that depend on mu) would need the initial state's own derivative added. */

/* Per-node shear modulus mu (n_box values in box order, device or host memory; values at
 * inactive nodes are ignored), replacing the material's mu (lambda is kept).  Needs
 * options.adjoint.  Takes effect at the next lbm_set_initial or step.  Errors: LBM_ERR_ARG,
 * LBM_ERR_STATE (no storage or options.adjoint not set), LBM_ERR_CUDA. */
int lbm_set_mu_field(lbm_handle *h, const double *mu);

/* Body force b (3 values, host memory), replacing options.body_force for later steps. */
int lbm_set_body_force(lbm_handle *h, const double *b);

/* Bytes of one saved state: populations, u*, u^n, the link reconstruction values and Newton
 * states, and the step counter.  A saved state restores the simulation exactly. */
int lbm_state_bytes(const lbm_handle *h, size_t *bytes);

/* Save the current state to / restore it from caller device memory (lbm_state_bytes bytes,
 * 256-byte aligned).  Enqueued on the handle's stream (a kernel writes the step counter);
 * lbm_load_state synchronises the stream to read the counter back.  Errors: LBM_ERR_ARG,
 * LBM_ERR_STATE (not initialised), LBM_ERR_CUDA. */
int lbm_save_state(lbm_handle *h, void *dst);
int lbm_load_state(lbm_handle *h, const void *src);

/* Bytes of one step's recorded moments (lbm_step_moments): the D*D components of F recovered in
 * that step (F - I in the FP32 form), one plane each over the padded box. */
int lbm_moments_bytes(const lbm_handle *h, size_t *bytes);

/* One step that also records its recovered F into `dst` (lbm_moments_bytes bytes, 256-byte
 * aligned, device memory) for lbm_adjoint_step.  Errors: LBM_ERR_ARG, LBM_ERR_STATE (not
 * initialised, or Neumann links present), LBM_ERR_CUDA. */
int lbm_step_moments(lbm_handle *h, void *dst);

/* Start a reverse sweep at the current state (after N steps): grad_u (D*n_box doubles in device
 * memory, box order) is dL/du at t_N for u = u* + dt/2 v as lbm_fields reports it.  Clears the
 * gradient accumulators.  Errors: LBM_ERR_ARG, LBM_ERR_STATE (not initialised, options.adjoint
 * not set, Neumann links present), LBM_ERR_CUDA. */
int lbm_adjoint_begin(lbm_handle *h, const double *grad_u);

/* Reverse one step: the k-th call after lbm_adjoint_begin reverses step N-k, and `moments` must
 * hold what lbm_step_moments recorded for that step (a recomputation from a saved state provides
 * it).  Accumulates the gradients.  Errors: LBM_ERR_ARG, LBM_ERR_STATE (no sweep in progress, or
 * all steps reversed), LBM_ERR_CUDA. */
int lbm_adjoint_step(lbm_handle *h, const void *moments);

/* Accumulated gradients: dL/dmu per box node (n_box doubles, device memory; zero at inactive
 * nodes) and dL/db (3 doubles, host memory); either may be null.  Synchronises. */
int lbm_adjoint_gradients(lbm_handle *h, double *grad_mu, double *grad_b);

/* Writes v, F (from U^num, Eq. state-recovery-general) and u = u* + dt/2 v
 * (Eq. u-recovery-general) at the current time.  Any pointer may be NULL.  Box planes
 * (LBM_LAYOUT_PLANES); the same as lbm_fields_ex(h, v, F, u, NULL, NULL, LBM_LAYOUT_PLANES). */
int lbm_fields(lbm_handle *h, double *v, double *F, double *u);

/* field layouts: PLANES component c of node n at c * n_box + n (structure of arrays); NODES at
 * n * ncomp + c (array of structures: a node's components contiguous) */
enum lbm_layout { LBM_LAYOUT_PLANES = 0, LBM_LAYOUT_NODES = 1 };

/* lbm_fields with the diagnostics of Algorithm 1's last loop: the Cauchy stress
 * sigma = J^-1 P F^T (Eq. cauchy-recovery-general; D*D components, row-major) and J = det F
 * (1 component), computed in FP64 from the recovered F.  Any pointer may be NULL; inactive nodes
 * are written as 0.  Device pointers, or host pointers with host staging.  Errors: LBM_ERR_ARG
 * (unknown layout, host pointer without staging), LBM_ERR_STATE (not initialised), LBM_ERR_CUDA. */
int lbm_fields_ex(lbm_handle *h, double *v, double *F, double *u, double *sigma, double *J, int layout);

/* Whole-body diagnostics of the current state (Sec. 5.2 reports the J range and the RMS velocity),
 * reduced on the GPU (warp shuffles, a fixed grid and a fixed order: the values do not depend on
 * the launch) over the active nodes:
 *   J_min, J_max    det F;
 *   v_rms, v_max    |v|;
 *   c_tangent       the largest tangent wave speed sqrt(max_n eig Q(n; F)) (Eq. acoustic-tensor-
 *                   general-d, rho0 = 1), the quantity the wave-speed audit bounds;
 *   incompat_rms    the compatibility residual of the projection's edge relation (Eq. projection-
 *                   edge-relation) for the current u and F, RMS over active axis edges of
 *                   |u_m - u_l - (F_m + F_l - 2I)(X_m - X_l)/2|, and n_edges the edge count.
 * Synchronises the stream.  Errors: LBM_ERR_ARG, LBM_ERR_STATE (not initialised), LBM_ERR_CUDA. */
typedef struct lbm_diag {
    double J_min, J_max, v_rms, v_max, c_tangent, incompat_rms;
    long long n_active, n_edges, step;
    double t;
} lbm_diag;
int lbm_diagnostics(lbm_handle *h, lbm_diag *out);

/* Synchronises the stream and reads (then clears) the device status word.
 * Returns LBM_ERR_DEVICE if it was non-zero, with the bits in *device_status. */
int lbm_sync(lbm_handle *h, int *device_status);

int lbm_get_info(const lbm_handle *h, lbm_info *info);

/* Per-kernel CUDA-event timing of lbm_step's launches (enable != 0 starts and
 * clears the accumulators); lbm_kernel_times synchronises and reports them. */
int lbm_enable_timing(lbm_handle *h, int enable);
int lbm_kernel_times(lbm_handle *h, lbm_kernel_time *out);

/* Cut-link geometry, for verification: copies n_cut entries into host arrays
 * (any may be NULL): node index, outgoing direction q (0:+x 1:-x 2:+y 3:-y
 * 4:+z 5:-z), eta, X_b (3 per link), N_b (3 per link), boundary id, LSQ
 * stencil size.  Synchronises the stream. */
int lbm_copy_links(lbm_handle *h, long long *node, int *q, double *eta, double *Xb, double *Nb, int *bid,
                   int *ns);

/* Active mask (1 byte per box node), for verification.  Synchronises. */
int lbm_copy_active(lbm_handle *h, unsigned char *mask);

void lbm_destroy(lbm_handle *h);
const char *lbm_error_string(int code);

/* Largest box (nodes) lbm_census_static accepts: 2^24, e.g. 256^3. */
#define LBM_CENSUS_MAX_NODES (1LL << 24)

/* Geometry census that allocates nothing.  No counterpart in the paper: it exists for
 * callers that must not allocate device memory when they size a simulation -- an embedding
 * runtime (a serving process, a solver framework) whose device memory is one arena planned ahead
 * and handed out by its own allocator, so that a library call must not take memory behind its
 * back, or a process already at its memory limit that must learn how much storage a body needs
 * before it can free or plan that much.  It returns the same counts that lbm_create computes
 * (lbm_info.n_active, n_cut, n_segments) for the grid and level set, which size the storage of
 * lbm_create and lbm_bind_storage, and applies lbm_create's domain rules.
 *
 * Scratch: one file-scope device array of 256 + LBM_CENSUS_MAX_NODES bytes (the active mask
 * and four counters), held by every GPU that loads the library until the process exits.
 * The first call on a device, with that device current, looks up the array's device address
 * (cudaGetSymbolAddress) and keeps it; make that first call before any stream capture.  All
 * calls on a device share the array, so calls that overlap on the GPU race; each call clears
 * the counters and rewrites the mask before use.  Work is enqueued on cuda_stream, then the
 * call synchronises that stream to return the counts.  It calls no cudaMalloc, cudaFree or
 * allocating library routine.
 * Takes single-body level sets of at most LBM_CENSUS_MAX_SHAPES shapes (ngroups must be 0).
 * Errors: LBM_ERR_ARG (invalid grid or level set, groups, too many shapes), LBM_ERR_CAPACITY
 * (more than LBM_CENSUS_MAX_NODES box nodes), LBM_ERR_DOMAIN (no active node, or the body extends
 * past a non-periodic box face; the counts are still written), LBM_ERR_CUDA. */
#define LBM_CENSUS_MAX_SHAPES 16
int lbm_census_static(const lbm_grid *grid, const lbm_levelset *levelset, void *cuda_stream, long long *n_active,
                      long long *n_cut, long long *n_segments);

#ifdef __cplusplus
}
#endif

#endif /* LBM_B300_H */
