/*
 * nmgb.h -- C ABI of the GB300 (sm_103a) library for the nodal finite-difference effective field and
 * Landau-Lifshitz-Gilbert integration of NeuralMag (Abert et al., arXiv 2411.11725).
 *
 * Model (section, equation labels of the paper):
 *   - Magnetisation m is a nodal vector field on a regular grid of N1 x N2 x N3 cuboid cells of size
 *     dx1 x dx2 x dx3 ("Nodal Finite-Difference Scheme", multi-indices c, n, i; Eq. nodal_basis).
 *   - Material parameters Ms, A, Ku are cell-wise constants (Eqs. ms_discrete, cell_basis).  A cell
 *     with Ms = 0 is vacuum and contributes to no term.
 *   - The effective field (Eq. heff) is the sum of exchange (Eq. exchange_energy), uniaxial
 *     anisotropy E = -int Ku (m.e)^2, Zeeman E = -mu0 int Ms h.m, each from its weak form (Eq.
 *     weak_form_discrete) assembled cell by cell (Eqs. weak_form_impl_f, weak_form_impl) and divided
 *     by the lumped nodal mass (Eq. mass_lumping); and the demagnetising field of homogeneously
 *     magnetised cuboid cells by zero-padded FFT convolution with node->cell and cell->node averaging
 *     (section "Demagnetization Field").  mu0 = 4 pi 1e-7.
 *   - LLG right-hand side: Eq. llg.  Integrators: classical RK4 and adaptive Dormand-Prince 5(4)
 *     (section "Automatic Differentiation and Time Integration").
 *
 * Layouts at this boundary (C order, component fastest, as the paper's tensors):
 *   nodal vector field  (N1+1, N2+1, N3+1, 3)
 *   cell scalar         (N1, N2, N3)
 *   cell vector         (N1, N2, N3, 3)
 *
 * Precision: NM_F32 evaluates h_eff (stencils, FFT demag, LLG right-hand side) in FP32 and keeps the
 * magnetisation, the RK error norm, step control and the Newell tensor set-up in FP64.  NM_F64 does
 * everything in FP64.  "real" below means float for NM_F32 meshes and double for NM_F64 meshes.
 *
 * Ownership: the caller owns every pointer it passes and may reuse it once the call returns (host
 * pointers) or once the mesh's stream has passed the call (device pointers).  The library owns the
 * mesh and its device workspaces.  Work is enqueued on the mesh's CUDA stream; calls that return host
 * values synchronise that stream.
 *
 * Errors: every entry point returns NM_OK (0) or a negative NM_ERR_* code and leaves a message for
 * nm_last_error() (thread-local).  No C++ exception crosses this boundary.  Arguments are validated
 * on the host before anything is enqueued.
 */
#ifndef NMGB_H
#define NMGB_H

#ifdef __cplusplus
extern "C" {
#endif

#define NM_OK 0
#define NM_ERR_ARG (-1)             /* invalid argument: shape, null pointer, non-positive size ... */
#define NM_ERR_OOM (-2)             /* device memory allocation failed */
#define NM_ERR_CUDA (-3)            /* a CUDA runtime call failed */
#define NM_ERR_STEP_UNDERFLOW (-4)  /* adaptive step size fell below dt_min or too many rejections */
#define NM_ERR_NONFINITE (-5)       /* non-finite values met where finite ones are required */
#define NM_ERR_TIMEOUT (-6)         /* a bounded wait ran out */
#define NM_ERR_STATE (-7)           /* call out of order, e.g. stepping before a state was set */

#define NM_F32 0  /* FP32 field evaluation, FP64 state and step control */
#define NM_F64 1  /* FP64 throughout */

/* effective-field terms (bit mask) */
#define NM_EXCH 1u
#define NM_ANIS 2u
#define NM_ZEE 4u
#define NM_DEMAG 8u
#define NM_ALL 15u
/* interfacial DMI (set with nm_set_dmi; not in NM_ALL).  A reading: the paper lists antisymmetric
 * exchange among the energies its scheme handles (section "Nodal Finite-Difference Scheme") without
 * giving one; this library takes E = int D [m_z div m - (m . grad) m_z] (interface normal along z). */
#define NM_DMI 16u
#define NM_TERMS_MASK 31u

/* integrators */
#define NM_RK4 1   /* classical Runge-Kutta, fixed step */
#define NM_DP54 2  /* Dormand-Prince 5(4), FSAL, adaptive */

/* nm_set_field kinds */
#define NM_FIELD_HEXT_UNIFORM 1  /* uniform applied field (A/m) */
#define NM_FIELD_HEXT_CELL 2     /* cell-wise applied field (A/m), cell vector layout */

/* memory spaces of state pointers */
#define NM_MEM_HOST 0
#define NM_MEM_DEVICE 1

typedef struct nm_mesh_s *nm_mesh;

/* Create a mesh of n1 x n2 x n3 cells of size dx1 x dx2 x dx3 (metres), precision NM_F32 or NM_F64,
 * working on the CUDA stream `cuda_stream` (a cudaStream_t; NULL = legacy default stream).
 * Supported sizes: 1 <= n1, n2 <= 1024 and 1 <= n3 <= 64 (padded transform lengths up to 2048 along x
 * and y and 128 along z); nm_footprint_bytes gives the device memory a size takes.
 * Allocates every device workspace the mesh needs, and encodes on the host the TMA descriptor that the
 * y passes of the demag transform use for their tiles of the spectrum buffer.  Errors: NM_ERR_ARG
 * (n_k < 1, a size beyond the supported range, dx_k <= 0, bad precision, out == NULL), NM_ERR_OOM,
 * NM_ERR_CUDA (a CUDA call failed, or the driver's descriptor encoder is unavailable or refused the
 * shape). */
int nm_create_mesh(int n1, int n2, int n3, double dx1, double dx2, double dx3, int precision,
                   void *cuda_stream, nm_mesh *out);

/* As nm_create_mesh, with the nodal basis chosen (section "Low-Dimensional Geometries"): basis 3 is the
 * trilinear basis of nm_create_mesh, (n1+1) x (n2+1) x (n3+1) nodes; basis 2 is the 2D nodal basis with
 * full 3D integration, (n1+1) x (n2+1) x 1 nodes whose basis functions are constant along z over all n3
 * cell layers (thin films: half the degrees of freedom of one cell layer); basis 1 is the 1D nodal basis
 * with full 3D integration, (n1+1) x 1 x 1 nodes whose basis functions are constant along y and z over
 * all n2 x n3 cells of the cross-section (wires).  Every nodal field of a basis-2 (basis-1) mesh has
 * shape (n1+1, n2+1, 1, 3) ((n1+1, 1, 1, 3)); cell fields keep all n2 x n3 cells.  The transpose product
 * and both adjoints (nm_h_eff_vjp, nm_adjoint_run, nm_adjoint_continuous) work on every basis: the
 * low-dimensional system is the trilinear one restricted to m constant along z (or y and z), and its
 * gradients are those of the restricted system.  The DMI term needs basis 3 (NM_ERR_ARG otherwise).
 * Errors: as nm_create_mesh; NM_ERR_ARG for a basis other than 1, 2 or 3. */
int nm_create_mesh_basis(int n1, int n2, int n3, double dx1, double dx2, double dx3, int precision, int basis,
                         void *cuda_stream, nm_mesh *out);

/* Release a mesh and all its device memory (synchronises its stream).  NULL is accepted. */
int nm_destroy_mesh(nm_mesh mesh);

/* Material (Eqs. ms_discrete, cell_basis): host FP64 cell scalars Ms (A/m), A (J/m), Ku (J/m^3); a
 * NULL array means the uniform value Ms0 / A0 / Ku0.  axis: host double[3], the uniaxial easy axis
 * (normalised here; must be non-zero).  alpha: Gilbert damping; gamma: reduced gyromagnetic ratio in
 * m/(A s) (Eq. llg).  Builds the lumped nodal mass (Eq. mass_lumping) and, on first call, the demag
 * tensor spectrum.  Errors: NM_ERR_ARG (negative Ms, zero axis, non-finite values), NM_ERR_CUDA. */
int nm_set_material(nm_mesh mesh, const double *Ms, double Ms0, const double *A, double A0,
                    const double *Ku, double Ku0, const double axis[3], double alpha, double gamma);

/* Applied field for the Zeeman term.  kind NM_FIELD_HEXT_UNIFORM: h(t) = amp * s(t), data ignored.
 * kind NM_FIELD_HEXT_CELL: h_c(t) = data_c * s(t) with data a host FP64 cell vector field (NULL
 * removes the cell field), amp ignored.  s(t) = 1 for freq_hz == 0, else sin(2 pi freq_hz t + phase).
 * The two kinds add up.  Errors: NM_ERR_ARG. */
int nm_set_field(nm_mesh mesh, int kind, const double *data, const double amp[3], double freq_hz,
                 double phase);

/* Resident state for the integrators: m (FP64 nodal vector field, host or device pointer per
 * `where`), time t, next step size dt.  Invalidates the FSAL slope.  The layout conversion counts
 * non-finite components on the device; such a state is refused with NM_ERR_NONFINITE and leaves the
 * mesh without a state (NM_ERR_STATE from the integrators until a valid state is set).  Synchronises.
 * Errors: NM_ERR_ARG, NM_ERR_NONFINITE, NM_ERR_CUDA. */
int nm_set_state(nm_mesh mesh, const double *m, int where, double t, double dt);

/* Copy the resident state out: m_out (FP64 nodal vector field, host or device per `where`; may be
 * NULL), t and dt (may be NULL).  Synchronises the stream. */
int nm_get_state(nm_mesh mesh, double *m_out, int where, double *t, double *dt);

/* Integrator options: renormalise |m| = 1 after each accepted step (default 1); smallest allowed
 * adaptive step dt_min (default 1e-22 s); consecutive rejections before NM_ERR_STEP_UNDERFLOW
 * (default 50). */
int nm_set_integrator(nm_mesh mesh, int renormalise, double dt_min, int max_rejections);

/* Arithmetic of the per-node terms of the Dormand-Prince error norm on FP32 meshes (the Dormand-Prince
 * integrator of the time-integration section; the norm and controller of nm_llg_step).  0 (default):
 * the terms (dt sum_i e_i k_i) / (atol + rtol max(|m|, |m5|)) are formed in FP32 from the FP32 slopes
 * and the FP32 copy of m, and summed in FP64.  1: every operation of the terms in FP64, from the same
 * FP32 slopes, the FP64 m and FP64 coefficients.  FP64 meshes always use FP64.  The FP32 terms carry
 * rounding of about 1e-7 of the largest slope contribution; the slopes themselves carry the FP32 field
 * error (about 1e-6 relative), so both settings estimate the same error to that accuracy.  The FP32
 * terms form sum_i e_i k_i as sum_{i>1} e_i (k_i - k_1) (the weights sum to zero), which keeps their
 * relative accuracy when the combination is far smaller than the slopes.  GB300's FP64 rate makes
 * setting 1 about ten times slower for this kernel (6.2 against 0.63 ms per step on 1024x1024x32
 * cells).  Errors: NM_ERR_ARG. */
int nm_set_error_norm(nm_mesh mesh, int fp64_terms);

/* Effective field h = H_eff(m) at time t for the terms in the mask (NM_EXCH|NM_ANIS|NM_ZEE|NM_DEMAG|NM_DMI):
 * m and h_out are DEVICE pointers to real nodal vector fields; m == NULL uses the resident state.
 * Nodes that touch no magnetic cell get h = 0.  Asynchronous, so the values of m are not checked: a
 * non-finite m gives a non-finite h (the demag convolution spreads it over the whole mesh).  Errors:
 * NM_ERR_ARG, NM_ERR_STATE (material not set), NM_ERR_CUDA. */
int nm_h_eff(nm_mesh mesh, const void *m, void *h_out, unsigned terms, double t);

/* Select the field terms used by the integrators (default NM_ALL; add NM_DMI for the DMI term). */
int nm_set_terms(nm_mesh mesh, unsigned terms);

/* Interfacial DMI constant (J/m^2): D is a HOST FP64 cell scalar field (N1, N2, N3), or NULL for the
 * uniform value D0.  The term enters the field and the integrators when NM_DMI is in the term mask:
 * its variation is assembled cell by cell from the element integrals int phi_i d_k phi_i' (k = x, y) of
 * the trilinear basis, like the exchange (Eqs. weak_form_impl_f, weak_form_impl), over magnetic cells,
 * and divided by the lumped mass.  Needs the 3D basis.  Errors: NM_ERR_ARG (non-finite values, a
 * mesh of basis 1 or 2), NM_ERR_OOM, NM_ERR_CUDA. */
int nm_set_dmi(nm_mesh mesh, const double *D, double D0);

/* One integrator step on the resident state.  NM_RK4 uses *dt as the fixed step; NM_DP54 attempts
 * *dt and on return *dt holds the proposed next step, *accepted tells whether the attempt was taken
 * (error norm <= 1 with tolerances rtol, atol).  *t is advanced on acceptance.  Synchronises.
 * Errors: NM_ERR_ARG, NM_ERR_STATE, NM_ERR_STEP_UNDERFLOW, NM_ERR_TIMEOUT (a demag pass's bounded wait
 * for its TMA tile copy ran out: not expected on a working GPU), NM_ERR_CUDA. */
int nm_llg_step(nm_mesh mesh, int method, double *t, double *dt, double rtol, double atol, int *accepted);

/* n_steps step attempts with no host round trip in between (step control runs on the device; the
 * step is replayed from a captured CUDA graph).  The resident t and dt are used and advanced.
 * Asynchronous: read results with nm_get_state or nm_get_counters. */
int nm_run_steps(nm_mesh mesh, int method, long n_steps, double rtol, double atol);

/* Volume-weighted mean of the resident m (weights: lumped nodal volume Σ_{c∋n} V/8 over magnetic cells),
 * the observable of the paper's standard-problem validation and of nm_run_until's samples.  out: HOST
 * FP64 array of 3.  Synchronises.  Errors: NM_ERR_ARG, NM_ERR_STATE, NM_ERR_CUDA. */
int nm_mean_m(nm_mesh mesh, double *out);

/* Accepted/rejected step counters and the last error norm (synchronises). Pointers may be NULL. */
int nm_get_counters(nm_mesh mesh, long *n_accepted, long *n_rejected, double *last_err);

/* Integrate the resident state to t_end.  NM_RK4 uses the fixed step dt0 (the last step is
 * shortened to land on t_end); NM_DP54 starts from dt0 (or the resident dt when dt0 <= 0).  When
 * sample_dt > 0, step ends are clipped to the sample times t0 + k sample_dt and the volume-weighted
 * mean of m (weights: lumped nodal volume) is written to samples_out[k*3 + j] (host FP64 array of
 * max_samples x 3) for k = 0 .. while t0 + k sample_dt <= t_end (k = 0 is the initial state).
 * n_accepted / n_rejected may be NULL.  Errors: NM_ERR_ARG, NM_ERR_STATE, NM_ERR_STEP_UNDERFLOW,
 * NM_ERR_TIMEOUT (as nm_llg_step), NM_ERR_CUDA. */
int nm_run_until(nm_mesh mesh, double t_end, int method, double rtol, double atol, double dt0,
                 double sample_dt, double *samples_out, long max_samples, long *n_accepted,
                 long *n_rejected);

/* Per-launch device times of one integrator step: the step's kernels are launched directly (not from
 * a graph) on the mesh's stream with CUDA events recorded after each launch, `reps` times on the
 * resident state (which advances).  Writes the mean milliseconds of launch i to ms_out[i] and its
 * name to names_out + 32*i (may be NULL), for i < min(*n_kernels, max_kernels).  Synchronises. */
int nm_profile_step(nm_mesh mesh, int method, int reps, double rtol, double atol, int max_kernels,
                    double *ms_out, char *names_out, int *n_kernels);

/* As nm_get_state with where = NM_MEM_HOST, but allocating nothing: the node-major staging copy of m
 * lives in a fixed 4 MiB device array of the library instead of a stream-ordered allocation.  The
 * paper has no counterpart; this serves callers that cannot allocate device memory when they read a
 * state back (a request loop whose HBM budget is fully committed to resident runs; a caller that keeps
 * allocator calls out of its read-back path).  m_out: HOST FP64 nodal vector field (or NULL for t, dt
 * only).  Limit: meshes of at most 174762 nodes (4 MiB / 24 B); larger meshes return NM_ERR_ARG.  The
 * first call on a device looks up the array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture on that device.  The address is kept per device together with the id
 * of the context it belongs to: after a reset of the device's primary context (cudaDeviceReset) the
 * next call looks it up again, so that first call after a reset should also precede any capture.
 * Nothing in the array needs to start at zero.  The
 * call synchronises the mesh's stream; calls on different meshes that overlap on the GPU (from several
 * host threads) race on the shared array.  Errors: NM_ERR_ARG, NM_ERR_STATE, NM_ERR_CUDA. */
int nm_get_state_noalloc(nm_mesh mesh, double *m_out, double *t, double *dt);

/* Transpose product of the effective field (the gradient of <v, h_eff(m)>), for inverse problems
 * (section "Inverse Micromagnetics"; static problems differentiate the discretised field, the
 * discretise-first approach).  m, v: DEVICE real nodal vector fields; grad_m (DEVICE real nodal vector
 * field) receives J_h(m)^T v; grad_Ms (DEVICE real cell scalar field, or NULL) receives the derivative
 * of <v, h_eff(m)> with respect to the cell Ms map (through the lumped mass, the Ms-weighted cell->node
 * averages and the demag source).  The applied field does not depend on m.  Asynchronous.
 * Errors: NM_ERR_ARG, NM_ERR_STATE, NM_ERR_OOM, NM_ERR_CUDA. */
int nm_h_eff_vjp(nm_mesh mesh, const void *m, const void *v, unsigned terms, double t, void *grad_m,
                 void *grad_Ms);

/* Integrate from the resident state to t_end (as nm_run_until) and return a sampled quadratic loss
 *   L = sum_k sum_{n,j} weight_{n,j} (m_{n,j}(t_k) - target_{n,j})^2
 * over the sample times t_k = t0 + k sample_dt <= t_end (k >= 1; k = 0 too when include_initial), or
 * over t_end alone when sample_dt <= 0, together with its exact discrete gradient: the adjoint of every
 * accepted step with the step sizes of the forward run frozen (backpropagation through the integrator,
 * section "Automatic Differentiation and Time Integration"), recomputing segments of
 * `checkpoint_every` steps from stored states (<= 0: 32).  weight, target: HOST FP64 nodal vector
 * fields (target may be NULL = 0).  Outputs (HOST FP64, each may be NULL except loss): loss; grad_Ms
 * (cell scalar field, dL/dMs); grad_m0 (nodal vector field, dL/dm(t0)); n_steps (accepted steps);
 * with grad_Ms, grad_m0 and grad_h all NULL only the forward run and its loss are computed;
 * grad_h (3 values: dL/dh of the uniform applied field amplitude of nm_set_field, the design variable of
 * the paper's field-angle inverse problem, section "Inverse Problems").
 * The resident state ends at t_end.  Synchronises.  Errors: as nm_run_until, NM_ERR_OOM. */
int nm_adjoint_run(nm_mesh mesh, int method, double t_end, double rtol, double atol, double dt0,
                   double sample_dt, const double *weight, const double *target, int include_initial,
                   long checkpoint_every, double *loss, double *grad_Ms, double *grad_m0, long *n_steps,
                   double *grad_h);

/* Continuous adjoint-state gradient (section "Inverse Micromagnetics", Eqs. adjoint_forward,
 * adjoint_objective and adjoint_system): n_steps classical Runge-Kutta steps of dt = (t_end - t0)/n_steps
 * from the resident state (t0) to t_end, the final-time loss
 *   L = sum_{n,j} weight_{n,j} (m_{n,j}(t_end) - target_{n,j})^2,
 * and then n_steps Runge-Kutta steps of -dt, backwards from t_end to t0, of the system
 *   dm/dt = f(t, m),  da/dt = -(df/dm)^T a,  du/dt = -(df/dtheta)^T a,
 *   m(t_end) = m_output,  a(t_end) = dL/dm(t_end),  u(t_end) = 0.
 * The trajectory is reconstructed by the backward integration, not stored, so the gradients carry the
 * reconstruction error (which shrinks with the fourth power of dt); nm_adjoint_run is the exact
 * gradient of the discrete forward map.  weight, target: HOST FP64 nodal vector fields (target may be
 * NULL = 0).  Outputs (HOST FP64, each may be NULL except loss): loss; grad_m0 = a(t0) (nodal vector
 * field); grad_Ms = u(t0) for the cell Ms map (cell scalar field); grad_h = u(t0) for the uniform
 * applied field amplitude (3 values); m0_rec = the reconstructed m(t0) (nodal vector field).  m is
 * renormalised after each step, forward and backward, as set by nm_set_integrator.  The resident state
 * ends at t_end.  Synchronises.  Errors: NM_ERR_ARG (n_steps < 1, t_end <= t0, NULL weight or loss),
 * NM_ERR_STATE (no material or state), NM_ERR_OOM, NM_ERR_CUDA. */
int nm_adjoint_continuous(nm_mesh mesh, double t_end, long n_steps, const double *weight, const double *target,
                          double *loss, double *grad_m0, double *grad_Ms, double *grad_h, double *m0_rec);

/* Arithmetic ceiling of the current GPU for the roofline of ALU-bound kernels (the paper has no
 * counterpart; it states the denominators of the FP64 path's roofline): a grid of independent fused
 * multiply-add chains filling every SM, `reps` launches timed with CUDA events.  kind 0: FP32, 1: FP64.
 * *flops_per_s receives 2 x the multiply-adds per second.  Synchronises.  Errors: NM_ERR_ARG,
 * NM_ERR_CUDA. */
int nm_measure_peak(int kind, int reps, double *flops_per_s);

/* Sizes of the mesh: nodes, cells, padded FFT lengths P1 P2 P3, and the device bytes the mesh holds. */
int nm_mesh_info(nm_mesh mesh, long *n_nodes, long *n_cells, int P[3], long *device_bytes);

/* Device bytes a mesh of this shape and precision would hold (for admission by HBM footprint). */
long nm_footprint_bytes(int n1, int n2, int n3, int precision);

/* Block until all work enqueued on the mesh's stream has finished. */
int nm_sync(nm_mesh mesh);

/* ------------------------------------------------------------------------------------------------
 * Serving: a request loop that runs many independent LLG integrations of different grid sizes and
 * materials on one GPU.  The paper has no serving layer; each run is the single-mesh integration above
 * (nm_run_until without samples) and its result is the same as that run alone.
 *
 * A server owns a worker thread and a pool of meshes.  Requests wait in a FIFO queue and are admitted
 * when a slot is free (at most max_active runs at once) and their mesh fits the HBM budget: the sum of
 * nm_footprint_bytes over the pooled meshes (running or idle) stays <= hbm_budget_bytes.  An idle mesh
 * of the request's shape, cell size and precision is reused (its tensor spectrum stays resident);
 * otherwise a mesh is created, with its tensor spectrum copied from a resident mesh of the same shape
 * when there is one, and idle meshes of other shapes are destroyed, least recently used first, to make
 * room.  Each admitted run keeps m and its RK state on the device and steps on its own stream in chunks
 * of captured step graphs with device-side step control, so runs overlap on the device; the worker only
 * reads each run's control block between chunks.  A request whose footprint exceeds the budget on its
 * own completes with status NM_ERR_OOM.
 * ------------------------------------------------------------------------------------------------ */
typedef struct nm_server_s *nm_server;

typedef struct {
    int n[3];             /* cells N1 N2 N3 */
    double dx[3];         /* cell size, m */
    int precision;        /* NM_F32 | NM_F64 */
    double Ms, A, Ku;     /* uniform material: A/m, J/m, J/m^3 */
    double axis[3];       /* anisotropy axis (normalised by the library) */
    double alpha, gamma;  /* damping; gyromagnetic ratio in m/(A s) */
    double h[3];          /* uniform applied field, A/m */
    unsigned terms;       /* NM_EXCH | NM_ANIS | NM_ZEE | NM_DEMAG */
    int method;           /* NM_RK4 | NM_DP54 */
    double t_end;         /* integrate from t = 0 to t_end, s */
    double rtol, atol;    /* DP5 tolerances */
    double dt0;           /* initial (RK4: fixed) step, s */
    const double *m0;     /* HOST FP64 nodal vector field; borrowed until the request's result is returned */
    double *m_out;        /* HOST FP64 nodal vector field receiving m(t_end), or NULL; borrowed likewise.
                             Page-locked memory makes the copy asynchronous to the worker. */
    long tag;             /* caller's identifier, echoed in the result */
} nm_request;

typedef struct {
    long tag;
    int status;                  /* NM_OK or the NM_ERR_* code of the failed run */
    long n_accepted, n_rejected; /* step attempts of the run */
    double t_final;              /* time reached */
    double queue_s;              /* submit -> admission, s */
    double run_s;                /* admission -> result ready, s */
    double latency_s;            /* submit -> result ready, s */
    int n_active_at_admit;       /* runs on the device when this one was admitted (itself included) */
    char message[128];           /* error message of a failed run ("" on success) */
} nm_result;

typedef struct {
    long submitted, completed, failed;
    int queued, active, pooled;  /* waiting requests; running runs; meshes held (running + idle) */
    int peak_active;
    long bytes_in_use;           /* sum of the footprints of the pooled meshes */
    long peak_bytes;
    long meshes_created, meshes_evicted, tensor_copies;
    double busy_s;               /* wall time with at least one run on the device */
    double active_s;             /* integral of the number of running runs over wall time */
    double wall_s;               /* since nm_server_create */
} nm_server_stats;

/* Start a server on the current CUDA device.  hbm_budget_bytes > 0; 1 <= max_active <= 256.
 * Errors: NM_ERR_ARG, NM_ERR_CUDA. */
int nm_server_create(long hbm_budget_bytes, int max_active, nm_server *out);

/* Queue a request (validated on the host; NM_ERR_ARG for bad sizes, tolerances or pointers; the cell
 * counts and limits of nm_create_mesh apply).  Thread-safe. */
int nm_server_submit(nm_server server, const nm_request *req);

/* Move up to max_results finished results into out (in completion order) and set *n_out; waits up to
 * wait_s seconds for the first one when none is ready (0: do not wait).  Thread-safe. */
int nm_server_poll(nm_server server, nm_result *out, int max_results, double wait_s, int *n_out);

/* Counters and occupancy of the server.  Thread-safe. */
int nm_server_stats_get(nm_server server, nm_server_stats *out);

/* Finish every queued and running request, stop the worker and free all meshes.  Results not yet
 * polled are dropped. */
int nm_server_destroy(nm_server server);

/* Message of the last failing call on this thread ("" if none). */
const char *nm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* NMGB_H */
