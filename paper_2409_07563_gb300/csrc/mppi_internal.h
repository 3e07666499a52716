// mppi_internal.h -- host-side context and the launch interfaces between the
// C ABI (api.cu) and the kernel translation units.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <utility>
#include <vector>

#include "../../include/mppi.h"

namespace mppi {

constexpr int kMaxNu = 8;
constexpr int kMaxNx = 16;
constexpr int kMaxTnu = 16384;
constexpr int kMaxK = 1 << 24;
constexpr int kUpdateThreads = 256;
constexpr int kUpdateQb = 2;          // Philox blocks (4 elements each) per update block
constexpr int kMaxUpdateChunks = 64;  // split-K factor cap of the update
constexpr int kUpdateCallsPerThread = 8;  // Philox calls per update thread before another chunk

// Device scratch owned by a context.
struct Scratch {
    float *S = nullptr;                 // [K] trajectory costs
    float *w = nullptr;                 // [K] weights of the listed samples (parallel to nz)
    int *nz = nullptr;                  // [K] samples with non-zero weight, in index order
    int *cand = nullptr;                // [2 (K + 256)] per-block weight candidates (k, S_k bits)
    float *partials = nullptr;          // [4 * max rollout blocks] (rho_b, eta_b, eta2_b, n_cand)
    float *upartials = nullptr;         // [kMaxUpdateChunks * Q * 4] update partial sums
    float *scalars = nullptr;           // [8] rho, eta, F, ess, valid, nnz, update-done
    unsigned int *tickets = nullptr;    // [4] last-block tickets (self-resetting)
    unsigned int *status = nullptr;     // [1] device status word
    unsigned long long *counter = nullptr;    // [1] step counter
    unsigned long long *last_step = nullptr;  // [1] step used by the latest mppi_step
    float *ckpt = nullptr;              // [nck][nx][K] states every ckpt_every steps (differentiable contexts)
    int ckpt_every = 0;
    float *io = nullptr;                // staging for mppi_step_host: x0, u_nom, u_new, stats
    float *saved_in = nullptr;          // x0 and u_nom of the latest step (differentiable contexts)
    float *adj = nullptr;               // adjoint scratch (allocated by the first backward)
    size_t adj_floats = 0;
};

// Everything a rollout / update launch needs, passed by value.
struct StepParams {
    int K, T, nx, nu;
    float dt, lambda, lam_beta;        // lam_beta = beta * lambda
    float gamma;                       // step size of the mean update (1: plain MPPI)
    int n_elite;                       // > 0: CEM elite-set weights instead of MPPI's
    float sigma[kMaxNu], ivar[kMaxNu];  // ivar = 1/sigma^2 (0 where sigma = 0)
    uint64_t seed;
    const float *x0, *u_nom;
    float *u_new, *weights_out, *stats_out, *costs_out;
    const float *dyn_params, *cost_params, *map;
    int n_dyn_params, n_cost_params, map_h, map_w;
    // scratch
    float *S, *partials, *upartials, *scalars;
    float *w;
    int *nz, *cand;
    float *saved_in;                    // non-null: block 0 of the rollout copies x0, u_nom here
    float *ckpt;                        // non-null: the rollout stores x_t of every sample here,
    int ckpt_every;                     //   [t / ckpt_every][nx][K], at t = 0, ckpt_every, ...
    unsigned int *tickets, *status;
    unsigned long long *counter, *last_step;
    int checked;                        // check computed indices (mppi_options.checked)
};

enum RolloutVariant {
    kVariantGeneric = 1,
    kVariantQuadGroup = 2,
    kVariantQuadPair = 4,
    kVariantMlpBf16 = 5,
    kVariantMlpF32 = 6,
    kVariantGenericPair = 7,
    kVariantMlpTc = 8
};

struct LaunchPlan {
    int variant = kVariantGeneric;
    int rollout_threads = 128;
    int rollout_blocks = 1;
    size_t rollout_smem = 0;
    int update_qtiles = 1;
    int update_chunks = 1;
    int update_chunk_len = 256;
};

}  // namespace mppi

// Event-pair record of kernel launches while profiling is on.
struct ProfileRecord {
    bool on = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> launches;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
};

struct mppi_ctx {
    int dyn_kind = 0, integrator = 0, nx = 0, nu = 0, cost_kind = 0;
    int K = 0, T = 0, beta = 1, precision = 0, block_threads = 0, variant_opt = 0, checked = 0;
    float dt = 0.f, lambda = 1.f;
    uint64_t seed = 0;
    std::vector<float> sigma, dyn_params_h, cost_params_h;
    std::vector<int> sphere_order;      // quadrotor crash test: neighbouring spheres paired
    float *d_dyn = nullptr, *d_cost = nullptr, *d_map = nullptr;
    int map_h = 0, map_w = 0;
    mppi::Scratch scr;
    float *io_host = nullptr;           // pinned, mapped staging for mppi_step_host (first use)
    float *io_host_dev = nullptr;       // its device address
    mppi::LaunchPlan plan;
    cudaStream_t stream = nullptr;
    int device = 0, num_sms = 0;
    bool have_step = false;
    bool differentiable = false;        // cart-pole + quadratic + Euler
    int iterations = 1;                 // Algorithm 1's outer loop
    float gamma = 1.f;                  // DMD-MPC step size of the mean update
    float *u_iter = nullptr;            // [2 T nu] means between iterations (iterations > 1)
    int n_elite = 0;                    // CEM elite-set size (0: MPPI weights)
    std::string err;
    ProfileRecord prof;
};

namespace mppi {

// Kernel translation units (rollout.cu, update.cu, ...).
bool rollout_supported(int dyn_kind, int cost_kind, int nx, int nu);
size_t rollout_smem_bytes(const mppi_ctx &c);
cudaError_t rollout_prepare(const mppi_ctx &c);  // sets smem attributes
cudaError_t launch_rollout(const mppi_ctx &c, const StepParams &p);
// the same models with a dynamics warp and a noise-and-cost warp per 32 samples
bool pair_rollout_applicable(const mppi_ctx &c);
size_t pair_rollout_smem_bytes(const mppi_ctx &c, int threads);
cudaError_t pair_rollout_prepare(const mppi_ctx &c);
cudaError_t launch_pair_rollout(const mppi_ctx &c, const StepParams &p);
cudaError_t launch_update(const mppi_ctx &c, const StepParams &p);
// the state trajectory of x0 under u (no noise): traj[(T+1) nx]
cudaError_t launch_nominal_trajectory(const mppi_ctx &c, const float *x0, const float *u,
                                      float *traj);
// out[t] = u[min(t + s, T - 1)]
cudaError_t launch_shift(const mppi_ctx &c, const float *u, int s, float *out);
// cem.cu: elite-set weights (list for the update kernel)
cudaError_t launch_cem_select(const mppi_ctx &c, const StepParams &p);
cudaError_t launch_sample_noise(uint64_t seed, uint64_t step, int K, int Q, uint32_t *bits,
                                float *z, cudaStream_t s);
cudaError_t launch_store_u64(unsigned long long *dst, unsigned long long v, cudaStream_t s);
// launch configuration with programmatic dependent launch (kernels start with
// a dependency wait, so consecutive step kernels overlap their launch)
cudaLaunchConfig_t pdl_config(dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              cudaLaunchAttribute *attr);
// adjoint.cu: backward of the cart-pole step
int adjoint_checkpoint_every(int T);                      // ceil(sqrt(T)), multiple of 4
size_t adjoint_checkpoint_floats(int K, int T, int nx);  // stored by every forward step
size_t adjoint_scratch_floats(int K, int T);
cudaError_t launch_adjoint(const mppi_ctx &c, const StepParams &sp, const float *G,
                           const float *u_nom, float *scratch, bool fresh, float *grad_out,
                           cudaStream_t s);
// rollout_quad.cu: four lanes per quadrotor sample
bool quad_group_applicable(const mppi_ctx &c);
size_t quad_group_smem_bytes(const mppi_ctx &c);
cudaError_t quad_group_prepare(const mppi_ctx &c);
cudaError_t launch_quad_group(const mppi_ctx &c, const StepParams &p);
// rollout_quad_pair.cu: one sample per thread, dynamics / cost / crash warps per 32 samples
bool quad_pair_applicable(const mppi_ctx &c);
int quad_pair_roles(const mppi_ctx &c);  // warps per 32 samples (4)
bool quad_pair_low_reg(const mppi_ctx &c);
void quad_pair_order_spheres(mppi_ctx &c);  // after every change of the cost parameters
size_t quad_pair_smem_bytes(const mppi_ctx &c, int threads);
cudaError_t quad_pair_prepare(const mppi_ctx &c);
cudaError_t launch_quad_pair(const mppi_ctx &c, const StepParams &p);
// rollout_mlp_bf16.cu: bicycle + MLP on the tensor cores
// rollout_mlp_tc.cu: bicycle + MLP with the MLP on tcgen05 tensor cores
// (128-sample tiles, accumulators in tensor memory)
size_t mlp_tc_smem_bytes(const mppi_ctx &c);
cudaError_t mlp_tc_prepare(const mppi_ctx &c);
cudaError_t launch_mlp_tc(const mppi_ctx &c, const StepParams &p);
size_t mlp_bf16_smem_bytes(const mppi_ctx &c, int threads);
cudaError_t mlp_bf16_prepare(const mppi_ctx &c);
cudaError_t launch_mlp_bf16(const mppi_ctx &c, const StepParams &p);
// rollout_mlp_f32.cu: bicycle + MLP in FP32, four lanes per sample
bool mlp_f32_applicable(const mppi_ctx &c);
size_t mlp_f32_smem_bytes(const mppi_ctx &c, int threads);
cudaError_t mlp_f32_prepare(const mppi_ctx &c);
cudaError_t launch_mlp_f32(const mppi_ctx &c, const StepParams &p);

}  // namespace mppi
