/*
 * llb.h -- C ABI of libllb, a GB300 (sm_103a) implementation of the
 * moment-only ("lightweight", "without populations") lattice Boltzmann
 * step of Tiribocchi et al., "Lightweight Lattice Boltzmann",
 * arXiv 2301.01622.
 *
 * What one step computes (Sec. II and III A of the paper): every node holds
 * only its hydrodynamic moments -- density rho, momentum j = rho u and the
 * momentum-flux tensor P (Eqs. (1)-(3)), ten fields for one component and eleven
 * for two.  A step reconstructs each neighbour's post-collision population
 * from that neighbour's moments (Eqs. (4)-(6) and (8)),
 * pull-streams it (Eq. (9), read as h_i(x, t+1) = h'_i[H(x - c_i, t)]),
 * and sums the streamed populations into the new moments (Eqs. (1)-(3)).  Two
 * flip-flop copies of the moment arrays hold times t and t+1 (Sec. III A).
 * Boundaries are periodic in x, y and z.
 *
 * Canonical moment layout (every host or device buffer that crosses this
 * ABI): field-major, x fastest, element (f, z, y, x) at index
 * ((f * nz + z) * ny + y) * nx + x, fields in the order
 *   one component : rho, j_x, j_y, j_z, P_xx, P_yy, P_zz, P_xy, P_xz, P_yz
 *   two components: rho1, rho2, j_x, j_y, j_z, P_xx, ..., P_yz
 * The moments are the pre-collision moments at integer time t.
 *
 * Ownership: the library owns the context and, unless the caller passes its
 * own device buffers in llb_params.buffers, the device state.  Host and device
 * buffers passed to the calls below stay owned by the caller; the library
 * copies from or into them and never keeps the pointer.
 *
 * Errors: every call returns LLB_OK (0) or a negative LLB_E* code; no C++
 * exception crosses the ABI.  A CUDA error inside a call makes the context
 * sticky-failed: every later call returns LLB_ESTATE until llb_destroy.
 * llb_last_error() returns a human-readable message for the last failure.
 *
 * Streams: all device work of a context is enqueued on llb_params.stream
 * (a cudaStream_t; NULL = the legacy default stream).  llb_step is
 * asynchronous; llb_get_moments, llb_diagnostics and llb_synchronize wait
 * for the stream.
 */
#ifndef LLB_H
#define LLB_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define LLB_API __attribute__((visibility("default")))
#else
#define LLB_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define LLB_OK         0
#define LLB_EINVAL    -1  /* bad argument (sizes, tau, lattice, pointer)   */
#define LLB_ENOMEM    -2  /* device or host allocation failed              */
#define LLB_ECUDA     -3  /* a CUDA runtime call or kernel launch failed   */
#define LLB_EUNSTABLE -4  /* non-finite value or rho <= 0 seen             */
#define LLB_ETIMEOUT  -5  /* a bounded device wait gave up                 */
#define LLB_ESTATE    -6  /* context unusable after an earlier CUDA error  */

/* ---- element types (storage on the device, and host/device buffers) -- */
#define LLB_F64 0   /* double                                              */
#define LLB_F32 1   /* float                                               */
/* 16-bit storage of the one-component moment-only state (llb_params.storage
 * only; host and device buffers crossing the ABI are LLB_F64 or LLB_F32).
 * The shifted moments d = rho - 1, j, A = P - cs^2 rho I are stored scaled
 * by 2^6, 2^4 and 2^10 and all arithmetic is FP32.                        */
#define LLB_F16S  2 /* IEEE binary16                                       */
#define LLB_BF16S 3 /* bfloat16                                            */

/* ---- schemes --------------------------------------------------------- */
/* The moment-only scheme of the paper (Sec. II-III A). */
#define LLB_SCHEME_MOMENT          0
/* Population-storing regularized LB: stores all Q populations (2Q for two
 * components: the total and colour-1 sets) and applies the same collision
 * (Eq. (8) on the projected moments; for two components the same forcing,
 * perturbation and recolouring) -- the same map as LLB_SCHEME_MOMENT in
 * exact arithmetic, used as the in-project baseline.  FP32 or FP64.       */
#define LLB_SCHEME_POPULATION      1
/* Population-storing plain BGK (Eq. (7) applied to the stored populations,
 * ghosts kept): the "standard LB with populations" of Sec. IV (for two
 * components the colour-gradient LB with populations of Sec. IV A).      */
#define LLB_SCHEME_POPULATION_BGK  2

/* ---- kernel choice for LLB_SCHEME_MOMENT ----------------------------- */
#define LLB_KERNEL_AUTO   0  /* fastest available for the shape            */
#define LLB_KERNEL_DIRECT 1  /* one thread per node, gathers Q neighbours  */
#define LLB_KERNEL_TILED  2  /* z-marching shared-memory tile kernel, plain loads */
#define LLB_KERNEL_TMA    3  /* same tile kernel, planes staged by TMA box loads  */

typedef struct llb_ctx llb_ctx;

typedef struct llb_params {
    int ncomp;        /* 1 (default) or 2 components                         */
    int storage;      /* LLB_F32 (default), LLB_F64, LLB_F16S, LLB_BF16S     */
    int scheme;       /* LLB_SCHEME_* (default LLB_SCHEME_MOMENT)            */
    int kernel;       /* LLB_KERNEL_* (default LLB_KERNEL_AUTO)              */
    int variant;      /* tuning variant, 0 = default.  One component, FP32:
                         tiled kernel 0..5 (TMA L2 prefetch, IEEE 1/rho,
                         64x8 and 32x8 tiles, split-phase plane barrier),
                         TMA kernel 0..2 (ring depth, tile); the other
                         storage types have one shape per kernel.  Two
                         components, FP32: 0..5 (tile 32x8 with approximate
                         FP32 quotients and a rolled plane loop; 64x4, 32x8,
                         32x16 with IEEE quotients; 32x8 approximate
                         unrolled; 64x4 approximate rolled).  A variant the
                         kernel does not have is LLB_EINVAL.  Every variant
                         computes the same step (to FP32 rounding)           */
    /* two-component colour-gradient / near-contact parameters (Sec. III A-B) */
    double beta;      /* recolouring strength, default 0.7                   */
    double A_s;       /* surface-tension (perturbation) strength, default 0.01 */
    double A_h;       /* near-contact repulsion strength, default 0.0        */
    double g_min;     /* |grad phi| below which the normal is zero, default 1e-6 */
    int h_c;          /* near-contact probe range in nodes, default 3        */
    void* stream;     /* cudaStream_t; NULL = legacy default stream          */
    /* Optional caller-owned device buffers for the two flip-flop copies of
     * the state, each at least llb_state_bytes() bytes and 256-byte aligned.
     * NULL = the library allocates (and frees) them.                       */
    void* buffers[2];
    /* Bound on any wait inside a kernel (TMA stage arrival), in milliseconds
     * of device clock; default 2000.  A wait that runs out makes the kernel
     * record an error, let its own copies in flight land (with the default
     * bound) and return; the next synchronising call reports LLB_ETIMEOUT.
     * Range 1..600000. */
    int wait_budget_ms;
    /* Test switches; 0 in normal use.  Bit 0 (fault injection): every TMA
     * stage barrier is armed for one byte more than its copy delivers, so no
     * stage wait can complete and every wait runs out after wait_budget_ms
     * (the copies themselves land normally; nothing faults).  Bit 1: the
     * two-component adjoint runs its first pass in the reference form, one
     * thread per node loading its neighbours' cotangents, instead of the
     * tiled kernel (same result up to rounding). */
    int debug_flags;
    /* Two components: 0 (default) takes the interface normal n = G/|G| only
     * where |G| >= g_min (n = 0 elsewhere).  eps > 0 takes the smooth norm
     * |G|_eps = sqrt(|G|^2 + eps^2) and n = G/|G|_eps at every node, with the
     * perturbation's trace term scaled by |n|^2 so that it still conserves
     * mass; the step is then differentiable (llb_adjoint of two components
     * requires it).  Not in the paper: a reading for gradients. */
    double grad_eps;
} llb_params;

typedef struct llb_diag {
    double mass[2];     /* sum of rho (one component) or of rho1, rho2     */
    double momentum[3]; /* sum of j                                        */
    double rho1_sum;    /* sum of rho (rho1 for two components) over nodes where it is > 0.5 */
    long long n_in;     /* number of such nodes                            */
    double rho1_avg;    /* rho1_sum / n_in (0 if n_in == 0): <rho>_{rho>0.5}, Sec. IV Fig. 2 */
    double min_rho;     /* minimum total density                           */
    int flags;          /* bit 0: non-finite value seen; bit 1: min_rho <= 0 */
    int reserved;
} llb_diag;

#define LLB_FLAG_NONFINITE   1
#define LLB_FLAG_NONPOSITIVE 2

typedef struct llb_footprint {
    int arrays;               /* whole-domain arrays held on the device, both flip-flop copies */
    int fields;               /* arrays per copy (10/11 moments, Q or 2Q populations) */
    size_t bytes_per_node;    /* state bytes per node, both copies           */
    size_t state_bytes;       /* bytes of one copy                           */
    size_t stream_bytes_per_node; /* algorithmic DRAM bytes per node per step (read + write) */
} llb_footprint;

/* Fill *p with the defaults listed in llb_params.  Never fails. */
LLB_API void llb_params_default(llb_params* p);

/* Storage accounting without touching a GPU (Sec. III A: 20 vs 38 arrays for
 * one component on D3Q19, 22 vs 76 for two).  p may be NULL (defaults).
 * Returns LLB_EINVAL on bad sizes or parameters. */
LLB_API int llb_footprint_query(int nx, int ny, int nz, int lattice, const llb_params* p,
                        llb_footprint* out);

/* Bytes of one state copy (what each of llb_params.buffers must hold).  The
 * moment-only state is stored with periodic ghost rows and columns, so this
 * is slightly more than fields * nodes * element size. */
LLB_API int llb_state_bytes(int nx, int ny, int nz, int lattice, const llb_params* p, size_t* out);

/* Create a context for an nx * ny * nz periodic box on the current CUDA
 * device.  lattice: 19 (D3Q19) or 27 (D3Q27).  tau: BGK relaxation time,
 * tau > 1/2 (viscosity nu = cs^2 (tau - 1/2), Sec. III B).  nx, ny, nz >= 1.
 * Two components need nx, ny, nz >= 4.  p may be NULL (defaults).
 * The state is zero until one of the llb_init_* calls.  On failure *out is
 * NULL and nothing is leaked. */
LLB_API int llb_create(llb_ctx** out, int nx, int ny, int nz, int lattice, double tau,
               const llb_params* p);

/* Release everything the context owns.  NULL-safe.  Waits for the stream. */
LLB_API void llb_destroy(llb_ctx* ctx);

/* Load canonical moments (layout above) from HOST memory of element type
 * host_dtype (LLB_F64 or LLB_F32).  Copies through a device staging buffer
 * and converts on the device.  Rejects rho <= 0 or non-finite input with
 * LLB_EUNSTABLE (checked on the device, the call synchronises; for two
 * components rho is the total density, and a colour density may be slightly
 * negative, as a stepped field's can be near interfaces).  Resets the
 * step counter to 0. */
LLB_API int llb_init_moments(llb_ctx* ctx, const void* host_m, int host_dtype);

/* Same, from DEVICE memory (e.g. a torch tensor), asynchronous, no check. */
LLB_API int llb_init_moments_device(llb_ctx* ctx, const void* dev_m, int dtype);

/* Initialise at local equilibrium, P = cs^2 rho I + rho u u (the second
 * moment of Eq. (5)), from HOST arrays: rho (ncomp fields: rho, or
 * rho1 then rho2) and u (3 fields), canonical layout, element type
 * host_dtype. */
LLB_API int llb_init_equilibrium(llb_ctx* ctx, const void* host_rho, const void* host_u, int host_dtype);

/* Advance nsteps >= 0 time steps (asynchronous on the context stream). */
LLB_API int llb_step(llb_ctx* ctx, int nsteps);

/* Same as llb_step, replayed from a CUDA graph: the first call for a given
 * nsteps (and flip-flop parity) captures the nsteps launches into a graph on
 * a private stream; later calls launch that graph on the context stream.
 * Saves the per-launch host overhead of long runs of short steps. */
LLB_API int llb_step_graph(llb_ctx* ctx, int nsteps);

/* Autotuner: times every kernel and tile/pipeline variant that can run this
 * context's shape (tiled, TMA, direct; `trials` launches each), keeps the
 * fastest and reports it through kernel/variant (either may be NULL).  The
 * state does not advance: each trial recomputes the current step into the
 * spare flip-flop copy.  Synchronises.  Population schemes are left as they
 * are. */
LLB_API int llb_autotune(llb_ctx* ctx, int trials, int* kernel, int* variant);

/* Copy the current canonical moments into caller HOST memory of element
 * type host_dtype.  Synchronises the stream. */
LLB_API int llb_get_moments(llb_ctx* ctx, void* host_out, int host_dtype);

/* Same into caller DEVICE memory, asynchronous. */
LLB_API int llb_get_moments_device(llb_ctx* ctx, void* dev_out, int dtype);

/* FP64 reductions of the current state (Sec. IV, Figs. 2, 5, 7 and mass /
 * momentum conservation).  Synchronises the stream. */
LLB_API int llb_diagnostics(llb_ctx* ctx, llb_diag* out);

/* Diagnostics of canonical one-component moments (rho, j, P; layout above)
 * that are already in DEVICE memory, with the same FP64 sums as
 * llb_diagnostics, for callers that cannot allocate device memory.  The
 * paper has no counterpart: this is a deployment convenience.
 *
 * Who needs it: frameworks that own the device allocator and forbid other
 * code from calling cudaMalloc, real-time loops that may not allocate on the
 * hot path (an allocation can block or fail at an arbitrary moment), and
 * embedders with a fixed device-memory budget.  This call allocates nothing:
 * no cudaMalloc, no cudaFree, no allocating library routine.  Its scratch is
 * a fixed 288 KB array in device memory that every GPU which loads the
 * library holds until the process exits.
 *
 * dev_m: nx*ny*nz*10 elements of type dtype (LLB_F32 or LLB_F64), caller-owned.
 * stream: cudaStream_t (NULL = legacy default stream).  host_out: caller-owned
 * host struct, filled before the call returns (the call copies the result to
 * it and synchronises the stream).  Limits: nx*ny*nz <= 67,108,864 nodes,
 * else LLB_EINVAL and nothing runs.  Every call shares the one scratch array
 * and each call overwrites the parts it reads, so nothing carries over from
 * an earlier call; calls whose work overlaps on the GPU (other streams, other
 * host threads) race on it and must be ordered by the caller.  The first call
 * on a device looks up the array's device address with that device current
 * and keeps it for the life of the process; make that first call before any
 * stream capture, and do not use the call across a cudaDeviceReset of that
 * device (the kept address then belongs to a context that no longer exists).
 * Returns LLB_OK, LLB_EINVAL or LLB_ECUDA. */
LLB_API int llb_diagnostics_noalloc(const void* dev_m, int dtype, int nx, int ny, int nz, void* stream,
                                    llb_diag* host_out);

/* Load canonical moments from HOST memory (element type host_dtype), advance
 * nsteps >= 1 time steps and write the canonical moments after the last
 * step into HOST memory: the same result as llb_init_moments + llb_step +
 * llb_get_moments, with the host<->device copies overlapped with the device
 * work.  The box is cut into slabs of whole z-planes; slab copies in,
 * per-slab steps (each waits for the input slabs its pull reaches) and slab
 * copies out run on three streams of the context, ordered by events, so the
 * call takes about as long as the larger of the two host copies.  With
 * nsteps > 1 only the first step overlaps the copies in and the last step
 * the copies out.  Moment-only contexts on the tiled kernels, one component
 * and two (for two components every slab is at least as thick as the planes
 * the phase-field gradient and the near-contact probes reach, 2 and 1 + h_c);
 * other contexts get the same result without the overlap.  Page-locked host
 * buffers let the copies run asynchronously.  host_in and host_out stay
 * owned by the caller and must not overlap.  Starts after the work already
 * queued on the context stream and synchronises.  Returns LLB_EUNSTABLE
 * (after the steps ran) if the input held rho <= 0 or a non-finite value. */
LLB_API int llb_step_host(llb_ctx* ctx, const void* host_in, void* host_out, int host_dtype, int nsteps);

/* Wait for all work of the context. */
LLB_API int llb_synchronize(llb_ctx* ctx);

/* Steps taken since the last llb_init_*. */
LLB_API int llb_steps_done(const llb_ctx* ctx, long long* out);

/* Device pointer of the current state copy, its element type and the kernel
 * the context runs (for profiling and zero-copy views).  Bit-for-bit
 * checkpoint: the current state copy (llb_state_bytes bytes: the shifted
 * moments in the context's padded layout, ghost copies included; field-major,
 * except the one-component FP32 state, which interleaves its ten fields per
 * block of 32 node positions), saved and
 * later written into the current state copy of a context created with the
 * same sizes and parameters (after its llb_init_*), resumes the run bit for
 * bit; llb_steps_done then counts from that restart. */
LLB_API int llb_state_device(const llb_ctx* ctx, void** dev_ptr, int* dtype, int* kernel);

/* Adjoint of nsteps moment-only steps (FP32 or FP64 state): the gradient of
 * a scalar loss L of the canonical moments after nsteps with respect to the
 * canonical moments at the start and to tau.  The context must hold the
 * starting state; it is restored before the call returns.
 * dev_gfinal: dL/dm(t + nsteps), 10 (one component) or 11 (two components)
 * canonical fields in device memory of element type dtype; dev_ginit:
 * receives dL/dm(t) (same layout and dtype); *dtau receives dL/dtau (may be
 * NULL).  The forward steps are run once with a checkpoint of the moments
 * every `every` steps (0 = round(sqrt(nsteps))) and each segment is
 * recomputed from its checkpoint during the backward sweep: ~nsteps/every +
 * every state copies of device memory, allocated during the call.  Two
 * components need A_h = 0 (the near-contact switch is not differentiable)
 * and grad_eps > 0 (the smooth interface normal).  Not in the paper (the
 * paper has no gradients).  Synchronises.  LLB_EINVAL for 16-bit states,
 * batch boxes, or two components without those two settings. */
LLB_API int llb_adjoint(llb_ctx* ctx, int nsteps, int every, const void* dev_gfinal, void* dev_ginit, int dtype,
                        double* dtau);

/* ---- batched ensembles ----------------------------------------------
 * Independent two-component boxes of (possibly) different sizes advanced
 * together: each step is ONE persistent launch whose CTAs walk the work
 * items of every box.  All boxes share lattice, tau and llb_params
 * (ncomp must be 2; p->stream is used for every box).  Not in the paper:
 * it serves ensembles of droplet collisions of the kind the paper's
 * "many drops" motivation (Sec. III B) calls for. */
typedef struct llb_batch llb_batch;

/* dims: 3 * ndomains ints, (nx, ny, nz) of each box (each >= 4). */
LLB_API int llb_batch_create(llb_batch** out, int ndomains, const int* dims, int lattice, double tau,
                             const llb_params* p);
/* Releases every box.  NULL-safe. */
LLB_API void llb_batch_destroy(llb_batch* b);
/* Borrow the context of box d for llb_init_*, llb_get_moments*,
 * llb_diagnostics; it stays owned by the batch (llb_step and llb_destroy on
 * it are refused / ignored). */
LLB_API int llb_batch_domain(llb_batch* b, int d, llb_ctx** ctx);
/* Total nodes over all boxes. */
LLB_API int llb_batch_nodes(const llb_batch* b, long long* nodes);
/* Advance every box by nsteps (one launch per step; asynchronous). */
LLB_API int llb_batch_step(llb_batch* b, int nsteps);
/* Same, replayed from a captured CUDA graph of nsteps launches. */
LLB_API int llb_batch_step_graph(llb_batch* b, int nsteps);
/* Time the tile variants (`trials` launches each, state unchanged), keep the
 * fastest, report it through *variant (may be NULL).  Synchronises. */
LLB_API int llb_batch_autotune(llb_batch* b, int trials, int* variant);

/* Bounds checks (library built with -DLLB_CHECKED, libllb_checked.so).
 * In that build every shared- and global-memory index of the stencil kernels
 * (moment-only one- and two-component, direct, TMA, batch, population) is
 * compared with its buffer's extent before the access; an access out of range
 * is skipped and the first one is recorded with a site code (1 exchange
 * write, 2 exchange read, 3 state load, 4 state store, 5 ghost store, 6 TMA
 * stage read, 7 phase-field read/write, 8 near-contact probe, 9 population
 * array).  This call synchronises the device, sets *enabled to 1 in the
 * checked build (0 in the normal one, where *site and *index are always 0),
 * and returns and clears the first record of each kernel file: *site = 0 when
 * nothing was out of range, else the site and the offending index.  Any
 * argument may be NULL.  Returns LLB_OK or LLB_ECUDA. */
LLB_API int llb_checked_status(int* enabled, int* site, long long* index);

/* Static strings; never NULL. */
LLB_API const char* llb_status_string(int status);
LLB_API const char* llb_last_error(const llb_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LLB_H */
