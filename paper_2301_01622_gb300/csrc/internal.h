// Internal context and launcher declarations of libllb (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>

#include "../../include/llb.h"
#include "layout.cuh"

struct llb_ctx {
    int nx = 0, ny = 0, nz = 0;
    int Q = 19;              // 19 or 27
    int ncomp = 1;
    int storage = LLB_F32;   // element type of the device state
    int scheme = LLB_SCHEME_MOMENT;
    int kernel = LLB_KERNEL_AUTO;  // resolved kernel (never AUTO after create)
    int variant = 0;               // tile/pipeline variant of the TMA kernel
    double tau = 1.0, omega = 1.0;
    llb_params params{};
    cudaStream_t stream = nullptr;
    int device = 0;
    int num_sms = 0;
    size_t N = 0;            // nodes
    int nf = 0;              // arrays per state copy
    size_t elem = 4;         // bytes per element of the state
    size_t state_bytes = 0;  // bytes of one state copy
    llb::Layout lay{};       // layout of moment-format buffers (state of the moment scheme,
                             // temporaries of the population schemes)
    CUtensorMap tmap[2];     // TMA stage-load descriptors of buf[0], buf[1] (TMA kernel)
    bool tmap_ok = false;
    CUtensorMap pmap[2];     // TMA L2-prefetch descriptors of buf[0], buf[1] (tiled kernel)
    bool pmap_ok = false;
    void* err_dev = nullptr; // device int: set by a kernel whose bounded wait gave up
    void* buf[2] = {nullptr, nullptr};
    bool owns[2] = {false, false};
    int cur = 0;             // buf[cur] holds the state at time t
    void* staging = nullptr; // canonical moments (FP64 worst case) for host/device conversion
    size_t staging_bytes = 0;
    void* diag_scratch = nullptr;  // per-block partial sums of the diagnostics
    void* phi_scratch = nullptr;   // phase field of the two-component population schemes (N elements)
    void* staging_out = nullptr;   // canonical output of the pipelined host step (llb_step_host)
    size_t staging_out_bytes = 0;
    cudaStream_t pipe[3] = {nullptr, nullptr, nullptr};  // copy-in, step, copy-out streams of llb_step_host
    size_t diag_scratch_bytes = 0;
    void* flag_dev = nullptr;      // device int for init-time checks
    long long t = 0;
    int sticky = LLB_OK;
    std::string msg;
    // persistent launch plans (grid sizes), 0 = kernel unusable for this shape
    int tile_ctas = 0;
    int tma_ctas = 0;
    // captured step sequences (llb_step_graph): one per starting flip-flop copy
    cudaGraphExec_t graph_exec[2] = {nullptr, nullptr};
    int graph_steps[2] = {0, 0};
    bool in_batch = false;   // owned by an llb_batch: stepped and destroyed by it
};

namespace llb {

size_t elem_size(int dtype);
int fields_of(const llb_ctx& c);           // arrays per state copy
int canonical_fields(const llb_ctx& c);    // 10 or 11

// Moment-only, one component (moment_step.cu, moment_tiled_*.cu, moment_tma.cu).
// in_index: which of the context's buffers is the input (selects the TMA map).
constexpr int kTiledVariants32 = 6;  // variants of the FP32 tiled kernel (other storage types: 1)
constexpr int kTmaVariants = 3;      // variants of the TMA kernel
cudaError_t launch_moment_direct(const llb_ctx& c, const void* in, void* out);
cudaError_t launch_moment_tiled(const llb_ctx& c, int in_index, const void* in, void* out);
// Output planes zlo .. zhi-1 only, on stream st (the pipelined host step).
cudaError_t launch_moment_tiled_range(const llb_ctx& c, int in_index, const void* in, void* out, int zlo, int zhi,
                                      cudaStream_t st);
cudaError_t launch_moment_tma(const llb_ctx& c, int in_index, void* out);
int moment_tiled_ctas(const llb_ctx& c);   // persistent grid size, 0 if the kernel cannot run
int moment_tma_ctas(const llb_ctx& c);
// Encode the TMA stage-load descriptor of a moment buffer; false if TMA cannot serve this shape.
bool moment_tma_encode(const llb_ctx& c, void* buf, CUtensorMap* out);
// Encode the L2-prefetch descriptor of the tiled kernel's box for a moment buffer.
bool moment_tiled_encode(const llb_ctx& c, void* buf, CUtensorMap* out);
// 4D (x, y, z, field) tensor map of a padded moment state, box_w x box_h nodes x 10 fields.
bool encode_box_map(const llb_ctx& c, void* buf, int box_w, int box_h, CUtensorMap* out);
// Per storage type (moment_tiled_<type>.cu)
int moment_tiled_ctas_f32(const llb_ctx& c);
int moment_tiled_ctas_f64(const llb_ctx& c);
int moment_tiled_ctas_f16(const llb_ctx& c);
int moment_tiled_ctas_bf16(const llb_ctx& c);
cudaError_t launch_moment_tiled_f32(const llb_ctx& c, int in_index, const void* in, void* out, int zlo, int zhi,
                                     cudaStream_t st);
cudaError_t launch_moment_tiled_f64(const llb_ctx& c, int in_index, const void* in, void* out, int zlo, int zhi,
                                     cudaStream_t st);
cudaError_t launch_moment_tiled_f16(const llb_ctx& c, int in_index, const void* in, void* out, int zlo, int zhi,
                                     cudaStream_t st);
cudaError_t launch_moment_tiled_bf16(const llb_ctx& c, int in_index, const void* in, void* out, int zlo, int zhi,
                                     cudaStream_t st);
void moment_tiled_box_f32(const llb_ctx& c, int* w, int* h);
void moment_tiled_box_f64(const llb_ctx& c, int* w, int* h);
void moment_tiled_box_f16(const llb_ctx& c, int* w, int* h);
void moment_tiled_box_bf16(const llb_ctx& c, int* w, int* h);

// Two-component colour-gradient moment-only step (cg_step.cu)
constexpr int kCGVariants = 6;  // tile / division variants of the two-component kernel
int cg_tiled_ctas(const llb_ctx& c);
cudaError_t launch_cg_tiled(const llb_ctx& c, const void* in, void* out);
// Output planes zlo .. zhi-1 on stream st.
cudaError_t launch_cg_tiled_range(const llb_ctx& c, const void* in, void* out, int zlo, int zhi, cudaStream_t st);

// One box of a batched ensemble: its state copies for this step and its items.
struct BatchDom {
    const void* in;
    void* out;
    Layout lay;
    int ncx, ntiles, zc, nitems;  // chunk-major schedule of the box
    int item_begin;               // first global item of the box
};
// Persistent grid size of the batch kernel (ctx gives lattice, storage, variant).
int cg_batch_ctas(const llb_ctx& c);
// Fill the schedule fields of d for box c (c.nx.. give the box size) and `grid` CTAs.
void cg_batch_plan(const llb_ctx& c, int grid, BatchDom* d);
// `next`: work-queue counter, zero at launch.
cudaError_t launch_cg_batch(const llb_ctx& c, const BatchDom* doms, int ndom, int total, int grid, int* next);

// Bounds-check records of the kernel translation units (checked build; the
// normal build reports none).  Read and clear; -1 if the copy fails.
int chk_take_tiled_f32(int* site, long long* index);
int chk_take_tiled_f64(int* site, long long* index);
int chk_take_tiled_f16(int* site, long long* index);
int chk_take_tiled_bf16(int* site, long long* index);
int chk_take_step(int* site, long long* index);
int chk_take_tma(int* site, long long* index);
int chk_take_cg(int* site, long long* index);
int chk_take_cg_batch(int* site, long long* index);
int chk_take_pop(int* site, long long* index);
int chk_take_adjoint(int* site, long long* index);

// Population-storing baselines (population_step.cu)
cudaError_t launch_population_step(const llb_ctx& c, const void* in, void* out, bool bgk);
// state <- populations reconstructed from shifted moments (un-streamed so a pull reads them)
cudaError_t launch_population_from_moments(const llb_ctx& c, const void* mom, void* state);
// shifted moments <- projection of the pulled populations
cudaError_t launch_moments_from_population(const llb_ctx& c, const void* state, void* mom);

// Conversions between canonical and shifted storage (convert.cu)
cudaError_t launch_canonical_to_shifted(const llb_ctx& c, const void* canon, int canon_dtype, void* state,
                                        int* bad_flag);
cudaError_t launch_shifted_to_canonical(const llb_ctx& c, const void* state, void* canon, int canon_dtype);
// One component: planes zlo .. zhi-1 only, on stream st.
cudaError_t launch_canonical_to_shifted_range(const llb_ctx& c, const void* canon, int canon_dtype, void* state,
                                              int* bad_flag, int zlo, int zhi, cudaStream_t st);
cudaError_t launch_shifted_to_canonical_range(const llb_ctx& c, const void* state, void* canon, int canon_dtype,
                                              int zlo, int zhi, cudaStream_t st);
cudaError_t launch_equilibrium(const llb_ctx& c, const void* rho, const void* u, int dtype, void* state,
                               int* bad_flag);

// Diagnostics (diagnostics.cu).  `mom` holds shifted moments of type c.storage.
int diag_blocks(const llb_ctx& c);
cudaError_t launch_diagnostics(const llb_ctx& c, const void* mom, void* scratch, llb_diag* dev_out);

}  // namespace llb
