// api.cu -- the C ABI declared in include/mppi.h: argument validation,
// context and scratch ownership, launch planning, and dispatch to the kernel
// translation units.  Every compute step runs in the kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "mppi_internal.h"

using mppi::StepParams;

namespace {

mppi_status fail(mppi_ctx *c, mppi_status st, const std::string &msg) {
    if (c) c->err = msg;
    return st;
}

mppi_status cuda_fail(mppi_ctx *c, cudaError_t e, const char *what) {
    return fail(c, e == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA,
                std::string(what) + ": " + cudaGetErrorString(e));
}

int expected_dyn_params(int kind, int nx, int nu) {
    switch (kind) {
    case MPPI_DYN_CARTPOLE: return 4;
    case MPPI_DYN_QUADROTOR: return 5;
    case MPPI_DYN_BICYCLE_MLP: return 1 + 64 * 6 + 64 + 64 * 64 + 64 + 4 * 64 + 4;
    case MPPI_DYN_DOUBLE_INTEGRATOR: return 0;
    case MPPI_DYN_LINEAR: return nx * nx + nx * nu;
    case MPPI_DYN_DIFF_DRIVE: return 4;
    default: return -1;
    }
}

bool fixed_dims(int kind, int &nx, int &nu) {
    switch (kind) {
    case MPPI_DYN_CARTPOLE: nx = 4; nu = 1; return true;
    case MPPI_DYN_QUADROTOR: nx = 13; nu = 4; return true;
    case MPPI_DYN_BICYCLE_MLP: nx = 7; nu = 2; return true;
    case MPPI_DYN_DOUBLE_INTEGRATOR: nx = 4; nu = 2; return true;
    case MPPI_DYN_DIFF_DRIVE: nx = 3; nu = 2; return true;
    default: return false;
    }
}

template <class T>
cudaError_t dalloc(T **p, size_t n) {
    return cudaMalloc(reinterpret_cast<void **>(p), std::max<size_t>(n, 1) * sizeof(T));
}

// Event pair around one launch while profiling is on (ordered on the stream).
class ProfScope {
  public:
    ProfScope(mppi_ctx *c, int slot) : c_(c), slot_(slot) {
        if (!c_->prof.on) return;
        a_ = take();
        b_ = take();
        if (a_ && b_) cudaEventRecord(a_, c_->stream);
    }
    ~ProfScope() {
        if (!c_->prof.on || !a_ || !b_) return;
        cudaEventRecord(b_, c_->stream);
        c_->prof.launches.push_back({slot_, {a_, b_}});
    }

  private:
    cudaEvent_t take() {
        auto &pr = c_->prof;
        if (pr.pool_used == pr.pool.size()) {
            cudaEvent_t e = nullptr;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            pr.pool.push_back(e);
        }
        return pr.pool[pr.pool_used++];
    }
    mppi_ctx *c_;
    int slot_;
    cudaEvent_t a_ = nullptr, b_ = nullptr;
};

void free_ctx(mppi_ctx *c) {
    if (!c) return;
    if (c->stream) cudaStreamSynchronize(c->stream);
    if (c->io_host) cudaFreeHost(c->io_host);
    if (c->u_iter) cudaFree(c->u_iter);
    for (cudaEvent_t e : c->prof.pool) cudaEventDestroy(e);
    void *ptrs[] = {c->d_dyn, c->d_cost, c->d_map, c->scr.S, c->scr.w, c->scr.nz, c->scr.cand,
                    c->scr.partials, c->scr.upartials,
                    c->scr.scalars, c->scr.tickets, c->scr.status, c->scr.counter,
                    c->scr.last_step, c->scr.ckpt, c->scr.io,
                    c->scr.saved_in, c->scr.adj};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete c;
}

void plan_launch(mppi_ctx &c) {
    mppi::LaunchPlan &pl = c.plan;
    const bool quad = mppi::quad_group_applicable(c) && c.variant_opt != mppi::kVariantGeneric;
    // Automatic: one sample per thread with four warp roles per 32 samples
    // (measured on GB300: 62.7 us per step at K = 8192, T = 150 against 70.6
    // for the four-lane warp pairs and 109 for the four-lane single warps;
    // 3.1e10 against 2.4e10 rollout-steps/s at K = 524288).
    const int asked = c.variant_opt == 0 ? mppi::kVariantQuadPair : c.variant_opt;
    const int roles = mppi::quad_pair_roles(c);  // warps per 32 samples
    const bool pair1 = quad && asked == mppi::kVariantQuadPair &&
                       c.block_threads % (32 * roles) == 0 && mppi::quad_pair_applicable(c);
    const bool group = quad && !pair1;
    const bool bf16 = c.precision == MPPI_PREC_BF16_MLP;
    // BF16 MLP: the warp-level mma.sync kernel by default (measured on GB300
    // at K = 16384, T = 100: 116 us against 198 for the tcgen05 kernel, whose
    // three dependent layers per step each wait for an MMA round trip);
    // rollout_variant 2 selects the tcgen05 kernel
    const bool mlp_tc = bf16 && c.variant_opt == mppi::kVariantQuadGroup;
    const bool mlp_sync = bf16 && !mlp_tc;
    const bool mlp32 = mppi::mlp_f32_applicable(c) && c.variant_opt != mppi::kVariantGeneric;
    const bool gpair = !bf16 && c.variant_opt == 0 && mppi::pair_rollout_applicable(c) &&
                       c.block_threads % 96 == 0 && c.block_threads <= 192;
    pl.variant = mlp_tc    ? mppi::kVariantMlpTc
                 : mlp_sync ? mppi::kVariantMlpBf16
                 : mlp32 ? mppi::kVariantMlpF32
                 : gpair ? mppi::kVariantGenericPair
                 : pair1 ? mppi::kVariantQuadPair
                 : group ? mppi::kVariantQuadGroup
                         : mppi::kVariantGeneric;
    // threads per sample (the FP32 MLP: four lanes per two samples)
    const int lanes = mlp_tc ? 3 : mlp_sync || mlp32 ? 2 : gpair ? 3 : pair1 ? roles : group ? 4 : 1;
    const long threads_needed = static_cast<long>(c.K) * lanes;
    if (mlp_tc) {
        pl.rollout_threads = 384;  // two 64-sample tiles: 2 x 4 tile warps, four cost warps
    } else if (c.block_threads > 0) {
        pl.rollout_threads = c.block_threads;
    } else if (mlp_sync) {
        // warp pairs of 32 samples spread over every SM first, at most four
        // per block: a block's warps occupy consecutive warp slots, so four
        // pairs put one dynamics warp on each SM sub-partition (measured on
        // GB300 at K = 16384, T = 100: 122 us per step against 166 for one
        // pair per block, whose dynamics warps share two sub-partitions)
        const long groups = (static_cast<long>(c.K) + 31) / 32;
        const long per_sm = (groups + c.num_sms - 1) / c.num_sms;
        pl.rollout_threads = 64 * static_cast<int>(std::min(4L, std::max(1L, per_sm)));
    } else if (gpair) {
        // warp triples spread over every SM first, at most two per block (two
        // blocks on an SM put their four dynamics warps on four sub-partitions;
        // K = 1024: 32 blocks of one triple)
        const long groups = (static_cast<long>(c.K) + 31) / 32;
        const long per_sm = (groups + c.num_sms - 1) / c.num_sms;
        pl.rollout_threads = 96 * static_cast<int>(std::min(2L, std::max(1L, per_sm)));
    } else if (mlp32) {
        // sixteen samples per warp; two warps per block once there are two
        // warps per SM (K = 16384: 512 blocks, about seven warps per SM)
        const long warps = (static_cast<long>(c.K) + 15) / 16;
        pl.rollout_threads = warps >= 2L * c.num_sms ? 64 : 32;
    } else if (pair1) {
        // warp groups of 32 samples spread over every SM first, at most two
        // groups per block (K = 8192: 256 groups, two per block on 128 SMs)
        const long groups = (static_cast<long>(c.K) + 31) / 32;
        const long per_sm = (groups + c.num_sms - 1) / c.num_sms;
        pl.rollout_threads = 32 * roles * static_cast<int>(std::min(2L, std::max(1L, per_sm)));
    } else if (group) {
        pl.rollout_threads = 64;
    } else {
        // Spread samples over every SM first (the rollout is a serial chain per
        // sample, so more SMs beat more warps per SM at these sizes).
        const int per_sm = (c.K + c.num_sms - 1) / c.num_sms;
        pl.rollout_threads = std::min(128, std::max(32, ((per_sm + 31) / 32) * 32));
    }
    pl.rollout_blocks = static_cast<int>((threads_needed + pl.rollout_threads - 1) / pl.rollout_threads);
    const int Q = c.nu * ((c.T + 3) / 4);
    pl.update_qtiles = (Q + mppi::kUpdateQb - 1) / mppi::kUpdateQb;
    const int max_chunks =
        std::min(mppi::kMaxUpdateChunks, (c.K + mppi::kUpdateThreads - 1) / mppi::kUpdateThreads);
    const int want = (2 * c.num_sms + pl.update_qtiles - 1) / pl.update_qtiles;
    pl.update_chunks = std::max(1, std::min(max_chunks, want));
    pl.update_chunk_len = (c.K + pl.update_chunks - 1) / pl.update_chunks;
}

StepParams make_params(const mppi_ctx &c) {
    StepParams p;
    std::memset(&p, 0, sizeof p);
    p.K = c.K;
    p.T = c.T;
    p.nx = c.nx;
    p.nu = c.nu;
    p.dt = c.dt;
    p.lambda = c.lambda;
    p.lam_beta = c.beta ? c.lambda : 0.f;
    p.gamma = c.gamma;
    p.n_elite = c.n_elite;
    for (int j = 0; j < c.nu; ++j) {
        p.sigma[j] = c.sigma[j];
        p.ivar[j] = c.sigma[j] > 0.f ? 1.0f / (c.sigma[j] * c.sigma[j]) : 0.f;
    }
    p.seed = c.seed;
    p.dyn_params = c.d_dyn;
    p.cost_params = c.d_cost;
    p.map = c.d_map;
    p.n_dyn_params = static_cast<int>(c.dyn_params_h.size());
    p.n_cost_params = static_cast<int>(c.cost_params_h.size());
    p.map_h = c.map_h;
    p.map_w = c.map_w;
    p.S = c.scr.S;
    p.w = c.scr.w;
    p.nz = c.scr.nz;
    p.cand = c.scr.cand;
    p.partials = c.scr.partials;
    p.upartials = c.scr.upartials;
    p.scalars = c.scr.scalars;
    p.tickets = c.scr.tickets;
    p.status = c.scr.status;
    p.counter = c.scr.counter;
    p.last_step = c.scr.last_step;
    p.saved_in = c.differentiable ? c.scr.saved_in : nullptr;
    p.ckpt = c.differentiable ? c.scr.ckpt : nullptr;
    p.ckpt_every = c.scr.ckpt_every;
    p.checked = c.checked;
    return p;
}

mppi_status validate_cost(const mppi_dynamics_desc &d, const mppi_cost_desc &cd, int nx, int nu,
                          std::string &msg) {
    if (cd.n_params > 0 && !cd.params) return msg = "cost params pointer is NULL", MPPI_ERR_INVALID_ARG;
    for (size_t i = 0; i < cd.n_params; ++i)
        if (!std::isfinite(cd.params[i]))
            return msg = "cost params must be finite", MPPI_ERR_INVALID_ARG;
    switch (cd.kind) {
    case MPPI_COST_QUADRATIC:
        if (cd.n_params != static_cast<size_t>(2 * nx + nu + 1))
            return msg = "QUADRATIC cost needs 2*nx+nu+1 params", MPPI_ERR_INVALID_ARG;
        return MPPI_OK;
    case MPPI_COST_QUAD_OBSTACLES: {
        if (d.kind != MPPI_DYN_QUADROTOR)
            return msg = "QUAD_OBSTACLES cost needs QUADROTOR dynamics", MPPI_ERR_UNSUPPORTED;
        if (cd.n_params < 33) return msg = "QUAD_OBSTACLES cost too short", MPPI_ERR_INVALID_ARG;
        const float nf = cd.params[31];
        const int n = static_cast<int>(nf);
        if (nf != static_cast<float>(n) || n < 0 || n > 256 ||
            cd.n_params != static_cast<size_t>(33 + 4 * n))
            return msg = "QUAD_OBSTACLES: n_obs must be an integer in [0,256] and the array "
                         "33 + 4*n_obs long",
                   MPPI_ERR_INVALID_ARG;
        return MPPI_OK;
    }
    case MPPI_COST_COSTMAP_SPEED:
        if (d.kind != MPPI_DYN_BICYCLE_MLP)
            return msg = "COSTMAP_SPEED cost needs BICYCLE_MLP dynamics", MPPI_ERR_UNSUPPORTED;
        if (cd.n_params != 6 || !cd.map || cd.map_h < 2 || cd.map_w < 2 || !(cd.params[5] > 0.f))
            return msg = "COSTMAP_SPEED needs 6 params (cell > 0) and a map of at least 2x2",
                   MPPI_ERR_INVALID_ARG;
        return MPPI_OK;
    case MPPI_COST_GOAL_COSTMAP:
        if (d.kind != MPPI_DYN_DIFF_DRIVE)
            return msg = "GOAL_COSTMAP cost needs DIFF_DRIVE dynamics", MPPI_ERR_UNSUPPORTED;
        if (cd.n_params != 9 || !cd.map || cd.map_h < 2 || cd.map_w < 2 || !(cd.params[8] > 0.f))
            return msg = "GOAL_COSTMAP needs 9 params (cell > 0) and a map of at least 2x2",
                   MPPI_ERR_INVALID_ARG;
        return MPPI_OK;
    case MPPI_COST_CIRCLE:
        if (d.kind != MPPI_DYN_DOUBLE_INTEGRATOR)
            return msg = "CIRCLE cost needs DOUBLE_INTEGRATOR dynamics", MPPI_ERR_UNSUPPORTED;
        if (cd.n_params != 7) return msg = "CIRCLE cost needs 7 params", MPPI_ERR_INVALID_ARG;
        return MPPI_OK;
    default:
        return msg = "unknown cost kind", MPPI_ERR_INVALID_ARG;
    }
}

}  // namespace

extern "C" {

void mppi_default_options(mppi_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof *opt);
    opt->beta = 1;
    opt->precision = MPPI_PREC_FP32;
}

mppi_status mppi_create(const mppi_dynamics_desc *dyn, const mppi_cost_desc *cost, int K, int T,
                        float dt, float lambda, const float *sigma, const mppi_options *opt,
                        mppi_ctx **out) {
    if (!out) return MPPI_ERR_INVALID_ARG;
    *out = nullptr;
    if (!dyn || !cost || !sigma) return MPPI_ERR_INVALID_ARG;
    mppi_options o;
    if (opt) o = *opt; else mppi_default_options(&o);

    int nx = dyn->nx, nu = dyn->nu;
    int fx, fu;
    if (fixed_dims(dyn->kind, fx, fu)) {
        if (nx != fx || nu != fu) return MPPI_ERR_INVALID_ARG;
    } else if (dyn->kind != MPPI_DYN_LINEAR) {
        return MPPI_ERR_INVALID_ARG;
    }
    if (nx < 1 || nx > mppi::kMaxNx || nu < 1 || nu > 4) return MPPI_ERR_INVALID_ARG;
    if (expected_dyn_params(dyn->kind, nx, nu) != static_cast<long>(dyn->n_params))
        return MPPI_ERR_INVALID_ARG;
    if (dyn->n_params > 0 && !dyn->params) return MPPI_ERR_INVALID_ARG;
    for (size_t i = 0; i < dyn->n_params; ++i)
        if (!std::isfinite(dyn->params[i])) return MPPI_ERR_INVALID_ARG;
    if (K < 1 || K > mppi::kMaxK || T < 1 || static_cast<long>(T) * nu > mppi::kMaxTnu)
        return MPPI_ERR_INVALID_ARG;
    if (!std::isfinite(dt) || !(dt > 0.f) || !std::isfinite(lambda) || !(lambda > 0.f))
        return MPPI_ERR_INVALID_ARG;
    for (int j = 0; j < nu; ++j)
        if (!std::isfinite(sigma[j]) || sigma[j] < 0.f) return MPPI_ERR_INVALID_ARG;
    if (o.beta != 0 && o.beta != 1) return MPPI_ERR_INVALID_ARG;
    if (o.checked != 0 && o.checked != 1) return MPPI_ERR_INVALID_ARG;
    if (o.block_threads < 0 || o.block_threads % 32 != 0 ||
        o.block_threads > 256)
        return MPPI_ERR_INVALID_ARG;
    if (o.rollout_variant < 0 || o.rollout_variant > 4) return MPPI_ERR_INVALID_ARG;
    // rollout_variant 3 (four lanes per sample with a dynamics and a cost warp
    // per eight samples) was retired: slower than the warp-role kernel
    if (o.rollout_variant == 3) return MPPI_ERR_UNSUPPORTED;
    if (o.rollout_variant == 4 && o.block_threads % 128 != 0) return MPPI_ERR_INVALID_ARG;
    if (o.precision == MPPI_PREC_BF16_MLP && o.block_threads % 64 != 0) return MPPI_ERR_INVALID_ARG;
    // the tcgen05 MLP kernel (rollout_variant 2) has one shape (384 threads per
    // 128 samples)
    const bool bf16_tc = o.precision == MPPI_PREC_BF16_MLP && o.rollout_variant == 2;
    if (bf16_tc && o.block_threads != 0) return MPPI_ERR_INVALID_ARG;
    if (o.precision == MPPI_PREC_BF16_MLP && o.rollout_variant > 2) return MPPI_ERR_UNSUPPORTED;
    if (o.rollout_variant >= 2 && !bf16_tc &&
        (dyn->kind != MPPI_DYN_QUADROTOR ||
         (cost->kind == MPPI_COST_QUAD_OBSTACLES && cost->n_params > 33 + 4 * 32)))
        return MPPI_ERR_UNSUPPORTED;
    const int want_integrator = dyn->kind == MPPI_DYN_QUADROTOR ? MPPI_RK4 : MPPI_EULER;
    if (dyn->integrator != MPPI_EULER && dyn->integrator != MPPI_RK4) return MPPI_ERR_INVALID_ARG;
    if (dyn->integrator != want_integrator) return MPPI_ERR_UNSUPPORTED;
    std::string msg;
    mppi_status st = validate_cost(*dyn, *cost, nx, nu, msg);
    if (st != MPPI_OK) return st;
    if (!mppi::rollout_supported(dyn->kind, cost->kind, nx, nu)) return MPPI_ERR_UNSUPPORTED;
    if (o.precision != MPPI_PREC_FP32 &&
        !(o.precision == MPPI_PREC_BF16_MLP && dyn->kind == MPPI_DYN_BICYCLE_MLP &&
          cost->kind == MPPI_COST_COSTMAP_SPEED))
        return MPPI_ERR_UNSUPPORTED;

    mppi_ctx *c = new (std::nothrow) mppi_ctx;
    if (!c) return MPPI_ERR_OOM;
    c->dyn_kind = dyn->kind;
    c->integrator = dyn->integrator;
    c->nx = nx;
    c->nu = nu;
    c->cost_kind = cost->kind;
    c->K = K;
    c->T = T;
    c->beta = o.beta;
    c->precision = o.precision;
    c->block_threads = o.block_threads;
    c->variant_opt = o.rollout_variant;
    c->checked = o.checked;
    c->dt = dt;
    c->lambda = lambda;
    c->seed = o.seed;
    c->sigma.assign(sigma, sigma + nu);
    c->dyn_params_h.assign(dyn->params, dyn->params + dyn->n_params);
    c->cost_params_h.assign(cost->params, cost->params + cost->n_params);
    if (c->dyn_kind == MPPI_DYN_QUADROTOR) mppi::quad_pair_order_spheres(*c);

    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device);
    if (e != cudaSuccess) {
        free_ctx(c);
        return MPPI_ERR_CUDA;
    }
    plan_launch(*c);
    c->differentiable = dyn->kind == MPPI_DYN_CARTPOLE && cost->kind == MPPI_COST_QUADRATIC &&
                        dyn->integrator == MPPI_EULER;
    if (c->differentiable) c->scr.ckpt_every = mppi::adjoint_checkpoint_every(T);

    const int Q = nu * ((T + 3) / 4);
    const size_t max_blocks = (4 * static_cast<size_t>(K) + 31) / 32;  // 32-thread blocks, 4 lanes

    const size_t io_floats = static_cast<size_t>(nx) + 2 * static_cast<size_t>(T) * nu + 4;
    if ((e = dalloc(&c->scr.S, K)) != cudaSuccess ||
        (e = dalloc(&c->scr.w, K)) != cudaSuccess ||
        (e = dalloc(&c->scr.nz, K)) != cudaSuccess ||
        (e = dalloc(&c->scr.cand, 2 * (static_cast<size_t>(K) + 256))) != cudaSuccess ||
        (e = dalloc(&c->scr.partials, 4 * max_blocks)) != cudaSuccess ||
        (e = dalloc(&c->scr.upartials, static_cast<size_t>(mppi::kMaxUpdateChunks) * Q * 4)) != cudaSuccess ||
        (e = dalloc(&c->scr.scalars, 8)) != cudaSuccess ||
        (e = dalloc(&c->scr.tickets, 4)) != cudaSuccess ||
        (e = dalloc(&c->scr.status, 1)) != cudaSuccess ||
        (e = dalloc(&c->scr.counter, 1)) != cudaSuccess ||
        (e = dalloc(&c->scr.last_step, 1)) != cudaSuccess ||
        (e = dalloc(&c->scr.io, io_floats)) != cudaSuccess ||
        (c->differentiable &&
         (e = dalloc(&c->scr.saved_in, static_cast<size_t>(nx) + static_cast<size_t>(T) * nu)) !=
             cudaSuccess) ||
        (c->differentiable &&
         (e = dalloc(&c->scr.ckpt, mppi::adjoint_checkpoint_floats(K, T, nx))) != cudaSuccess) ||
        (e = dalloc(&c->d_dyn, c->dyn_params_h.size())) != cudaSuccess ||
        (e = dalloc(&c->d_cost, c->cost_params_h.size())) != cudaSuccess) {
        free_ctx(c);
        return e == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA;
    }
    if (cost->kind == MPPI_COST_COSTMAP_SPEED || cost->kind == MPPI_COST_GOAL_COSTMAP) {
        c->map_h = cost->map_h;
        c->map_w = cost->map_w;
        const size_t n = static_cast<size_t>(cost->map_h) * cost->map_w;
        if ((e = dalloc(&c->d_map, n)) != cudaSuccess ||
            (e = cudaMemcpy(c->d_map, cost->map, n * sizeof(float), cudaMemcpyHostToDevice)) != cudaSuccess) {
            free_ctx(c);
            return e == cudaErrorMemoryAllocation ? MPPI_ERR_OOM : MPPI_ERR_CUDA;
        }
    }
    if ((e = cudaMemcpy(c->d_dyn, c->dyn_params_h.data(), c->dyn_params_h.size() * sizeof(float),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(c->d_cost, c->cost_params_h.data(), c->cost_params_h.size() * sizeof(float),
                        cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemset(c->scr.tickets, 0, 4 * sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaMemset(c->scr.status, 0, sizeof(unsigned int))) != cudaSuccess ||
        (e = cudaMemset(c->scr.counter, 0, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMemset(c->scr.last_step, 0, sizeof(unsigned long long))) != cudaSuccess ||
        (e = cudaMemset(c->scr.scalars, 0, 7 * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(c->scr.scalars + 7, 0xff, sizeof(float))) != cudaSuccess) {  // running min
        free_ctx(c);
        return MPPI_ERR_CUDA;
    }
    c->plan.rollout_smem =
        c->plan.variant == mppi::kVariantQuadGroup ? mppi::quad_group_smem_bytes(*c)
        : c->plan.variant == mppi::kVariantQuadPair ? mppi::quad_pair_smem_bytes(*c, c->plan.rollout_threads)
        : c->plan.variant == mppi::kVariantMlpBf16 ? mppi::mlp_bf16_smem_bytes(*c, c->plan.rollout_threads)
        : c->plan.variant == mppi::kVariantMlpTc ? mppi::mlp_tc_smem_bytes(*c)
        : c->plan.variant == mppi::kVariantMlpF32 ? mppi::mlp_f32_smem_bytes(*c, c->plan.rollout_threads)
        : c->plan.variant == mppi::kVariantGenericPair ? mppi::pair_rollout_smem_bytes(*c, c->plan.rollout_threads)
                                                   : mppi::rollout_smem_bytes(*c);
    int max_smem = 0;
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device);
    if (c->plan.rollout_smem > static_cast<size_t>(max_smem)) {
        free_ctx(c);
        return MPPI_ERR_UNSUPPORTED;
    }
    if ((e = mppi::rollout_prepare(*c)) != cudaSuccess ||
        (c->plan.variant == mppi::kVariantQuadGroup && (e = mppi::quad_group_prepare(*c)) != cudaSuccess) ||
        (c->plan.variant == mppi::kVariantQuadPair && (e = mppi::quad_pair_prepare(*c)) != cudaSuccess) ||
        (c->plan.variant == mppi::kVariantMlpBf16 && (e = mppi::mlp_bf16_prepare(*c)) != cudaSuccess) ||
        (c->plan.variant == mppi::kVariantMlpTc && (e = mppi::mlp_tc_prepare(*c)) != cudaSuccess) ||
        (c->plan.variant == mppi::kVariantMlpF32 && (e = mppi::mlp_f32_prepare(*c)) != cudaSuccess) ||
        (c->plan.variant == mppi::kVariantGenericPair && (e = mppi::pair_rollout_prepare(*c)) != cudaSuccess)) {
        free_ctx(c);
        return MPPI_ERR_CUDA;
    }
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) {
        free_ctx(c);
        return MPPI_ERR_CUDA;
    }
    *out = c;
    return MPPI_OK;
}

void mppi_destroy(mppi_ctx *ctx) { free_ctx(ctx); }

mppi_status mppi_set_stream(mppi_ctx *ctx, void *cuda_stream) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    ctx->stream = static_cast<cudaStream_t>(cuda_stream);
    return MPPI_OK;
}

mppi_status mppi_step(mppi_ctx *ctx, const float *x0_d, const float *u_nom_d, float *u_new_d,
                      float *weights_d, float *stats_d, float *costs_d) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    if (!x0_d || !u_nom_d || !u_new_d)
        return fail(ctx, MPPI_ERR_INVALID_ARG, "x0, u_nom and u_new must be device pointers");
    const size_t TN = static_cast<size_t>(ctx->T) * ctx->nu;
    // Algorithm 1's outer loop: round i samples around the mean of round
    // i - 1 (ping-pong through u_iter); only the last round writes the
    // caller's outputs.  The kernels advance the step counter once per round.
    for (int it = 0; it < ctx->iterations; ++it) {
        const bool last = it == ctx->iterations - 1;
        StepParams p = make_params(*ctx);
        p.x0 = x0_d;
        p.u_nom = it == 0 ? u_nom_d : ctx->u_iter + ((it - 1) & 1) * TN;
        p.u_new = last ? u_new_d : ctx->u_iter + (it & 1) * TN;
        p.weights_out = last ? weights_d : nullptr;
        p.stats_out = last ? stats_d : nullptr;
        p.costs_out = last ? costs_d : nullptr;
        cudaError_t e;
        {
            ProfScope ps(ctx, MPPI_PROF_ROLLOUT);
            e = ctx->plan.variant == mppi::kVariantQuadGroup ? mppi::launch_quad_group(*ctx, p)
                : ctx->plan.variant == mppi::kVariantQuadPair ? mppi::launch_quad_pair(*ctx, p)
                : ctx->plan.variant == mppi::kVariantMlpBf16 ? mppi::launch_mlp_bf16(*ctx, p)
                : ctx->plan.variant == mppi::kVariantMlpTc ? mppi::launch_mlp_tc(*ctx, p)
                : ctx->plan.variant == mppi::kVariantMlpF32 ? mppi::launch_mlp_f32(*ctx, p)
                : ctx->plan.variant == mppi::kVariantGenericPair ? mppi::launch_pair_rollout(*ctx, p)
                                                             : mppi::launch_rollout(*ctx, p);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "rollout launch");
        if (ctx->n_elite > 0) {  // CEM: the elite set replaces the MPPI weights
            ProfScope ps(ctx, MPPI_PROF_OTHER);
            e = mppi::launch_cem_select(*ctx, p);
            if (e != cudaSuccess) return cuda_fail(ctx, e, "elite-set launch");
        }
        {
            ProfScope ps(ctx, MPPI_PROF_UPDATE);
            e = mppi::launch_update(*ctx, p);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "update launch");
    }
    ctx->have_step = true;
    ctx->err.clear();
    return MPPI_OK;
}

mppi_status mppi_step_host(mppi_ctx *ctx, const float *x0_h, const float *u_nom_h,
                           float *u_new_h, float *stats_h) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    if (!x0_h || !u_nom_h || !u_new_h)
        return fail(ctx, MPPI_ERR_INVALID_ARG, "x0, u_nom and u_new must be host pointers");
    const size_t TN = static_cast<size_t>(ctx->T) * ctx->nu, nx = static_cast<size_t>(ctx->nx);
    // pinned, device-mapped staging [x0 | u_nom | u_new | stats]: one copy of
    // the inputs into device memory (every block reads them), and the update
    // writes u_new and the statistics straight into the mapped host buffer
    // (measured on GB300: 77 against 86 us per quadrotor step with a second,
    // device-to-host copy)
    float *d_x0 = ctx->scr.io, *d_u = d_x0 + nx;
    cudaError_t e;
    if (!ctx->io_host) {
        if ((e = cudaHostAlloc(reinterpret_cast<void **>(&ctx->io_host),
                               sizeof(float) * (nx + 2 * TN + 4), cudaHostAllocMapped)) !=
            cudaSuccess) {
            ctx->io_host = nullptr;
            return cuda_fail(ctx, e, "pinned staging allocation");
        }
        if ((e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&ctx->io_host_dev),
                                          ctx->io_host, 0)) != cudaSuccess) {
            cudaFreeHost(ctx->io_host);
            ctx->io_host = nullptr;
            return cuda_fail(ctx, e, "mapped staging pointer");
        }
    }
    float *h = ctx->io_host, *hd = ctx->io_host_dev;
    std::memcpy(h, x0_h, nx * sizeof(float));
    std::memcpy(h + nx, u_nom_h, TN * sizeof(float));
    if ((e = cudaMemcpyAsync(d_x0, h, (nx + TN) * sizeof(float), cudaMemcpyHostToDevice,
                             ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "host-to-device copy");
    mppi_status st = mppi_step(ctx, d_x0, d_u, hd + nx + TN, nullptr, hd + nx + 2 * TN, nullptr);
    if (st != MPPI_OK) return st;
    if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess)
        return cuda_fail(ctx, e, "stream synchronize");
    std::memcpy(u_new_h, h + nx + TN, TN * sizeof(float));
    if (stats_h) std::memcpy(stats_h, h + nx + 2 * TN, 4 * sizeof(float));
    return MPPI_OK;
}

mppi_status mppi_set_params_device(mppi_ctx *ctx, const float *dyn_params_d,
                                   const float *cost_params_d) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    if (cost_params_d && ctx->dyn_kind == MPPI_DYN_QUADROTOR)
        return fail(ctx, MPPI_ERR_UNSUPPORTED,
                    "quadrotor cost constants are staged from the host copy: use mppi_set_params");
    cudaError_t e = cudaSuccess;
    if (dyn_params_d)
        e = cudaMemcpyAsync(ctx->d_dyn, dyn_params_d, ctx->dyn_params_h.size() * sizeof(float),
                            cudaMemcpyDeviceToDevice, ctx->stream);
    if (e == cudaSuccess && cost_params_d)
        e = cudaMemcpyAsync(ctx->d_cost, cost_params_d, ctx->cost_params_h.size() * sizeof(float),
                            cudaMemcpyDeviceToDevice, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "parameter copy");
    return MPPI_OK;
}

mppi_status mppi_set_params(mppi_ctx *ctx, const float *dyn_params, const float *cost_params) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    if (dyn_params) {
        for (size_t i = 0; i < ctx->dyn_params_h.size(); ++i)
            if (!std::isfinite(dyn_params[i]))
                return fail(ctx, MPPI_ERR_INVALID_ARG, "dynamics params must be finite");
        ctx->dyn_params_h.assign(dyn_params, dyn_params + ctx->dyn_params_h.size());
        e = cudaMemcpy(ctx->d_dyn, ctx->dyn_params_h.data(),
                       ctx->dyn_params_h.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "parameter upload");
    }
    if (cost_params) {
        for (size_t i = 0; i < ctx->cost_params_h.size(); ++i)
            if (!std::isfinite(cost_params[i]))
                return fail(ctx, MPPI_ERR_INVALID_ARG, "cost params must be finite");
        if (ctx->cost_kind == MPPI_COST_QUAD_OBSTACLES && cost_params[31] != ctx->cost_params_h[31])
            return fail(ctx, MPPI_ERR_INVALID_ARG, "the obstacle count cannot change");
        ctx->cost_params_h.assign(cost_params, cost_params + ctx->cost_params_h.size());
        if (ctx->dyn_kind == MPPI_DYN_QUADROTOR) mppi::quad_pair_order_spheres(*ctx);
        e = cudaMemcpy(ctx->d_cost, ctx->cost_params_h.data(),
                       ctx->cost_params_h.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "parameter upload");
    }
    return MPPI_OK;
}

mppi_status mppi_step_backward(mppi_ctx *ctx, const float *grad_u_new_d, float *grad_params_d) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    if (!ctx->differentiable)
        return fail(ctx, MPPI_ERR_UNSUPPORTED,
                    "backward needs CARTPOLE dynamics, QUADRATIC cost and EULER");
    if (!ctx->have_step) return fail(ctx, MPPI_ERR_UNSUPPORTED, "backward needs a prior mppi_step");
    if (ctx->iterations != 1 || ctx->gamma != 1.f || ctx->n_elite != 0)
        return fail(ctx, MPPI_ERR_UNSUPPORTED,
                    "backward differentiates one plain MPPI iteration (iterations 1, step size 1, "
                    "no CEM)");
    if (!grad_u_new_d || !grad_params_d)
        return fail(ctx, MPPI_ERR_INVALID_ARG, "grad_u_new and grad_params must be device pointers");
    cudaError_t e;
    const size_t need = mppi::adjoint_scratch_floats(ctx->K, ctx->T);
    const bool fresh = ctx->scr.adj_floats < need;
    if (fresh) {
        if (ctx->scr.adj) cudaFree(ctx->scr.adj);
        ctx->scr.adj = nullptr;
        ctx->scr.adj_floats = 0;
        if ((e = dalloc(&ctx->scr.adj, need)) != cudaSuccess)
            return cuda_fail(ctx, e, "adjoint scratch allocation");
        ctx->scr.adj_floats = need;
    }
    StepParams p = make_params(*ctx);
    {
        ProfScope ps(ctx, MPPI_PROF_ADJOINT);
        e = mppi::launch_adjoint(*ctx, p, grad_u_new_d, ctx->scr.saved_in + ctx->nx,
                                 ctx->scr.adj, fresh, grad_params_d, ctx->stream);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "adjoint launch");
    return MPPI_OK;
}

mppi_status mppi_set_iterations(mppi_ctx *ctx, int iterations, float step_size) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    if (iterations < 1 || iterations > 1024 || !std::isfinite(step_size) || !(step_size >= 0.f))
        return fail(ctx, MPPI_ERR_INVALID_ARG, "iterations 1..1024 and a finite step size >= 0");
    if (iterations > 1 && !ctx->u_iter) {
        cudaError_t e = dalloc(&ctx->u_iter, 2 * static_cast<size_t>(ctx->T) * ctx->nu);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "iteration scratch allocation");
    }
    ctx->iterations = iterations;
    ctx->gamma = step_size;
    return MPPI_OK;
}

mppi_status mppi_set_cem(mppi_ctx *ctx, float top_k_fraction) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    if (!std::isfinite(top_k_fraction) || top_k_fraction < 0.f || top_k_fraction > 1.f)
        return fail(ctx, MPPI_ERR_INVALID_ARG, "top_k_fraction in [0, 1]");
    if (top_k_fraction == 0.f) {
        ctx->n_elite = 0;
        return MPPI_OK;
    }
    const double n = std::floor(static_cast<double>(ctx->K) * static_cast<double>(top_k_fraction));
    ctx->n_elite = std::max(1, static_cast<int>(n));
    return MPPI_OK;
}

mppi_status mppi_nominal_trajectory(mppi_ctx *ctx, const float *x0_d, const float *u_d,
                                    float *traj_d) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    if (!x0_d || !u_d || !traj_d)
        return fail(ctx, MPPI_ERR_INVALID_ARG, "x0, u and traj must be device pointers");
    cudaError_t e = mppi::launch_nominal_trajectory(*ctx, x0_d, u_d, traj_d);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "trajectory launch");
    return MPPI_OK;
}

mppi_status mppi_shift(mppi_ctx *ctx, const float *u_d, int s, float *out_d) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    if (!u_d || !out_d || s < 0)
        return fail(ctx, MPPI_ERR_INVALID_ARG, "u and out must be device pointers, s >= 0");
    const size_t TN = static_cast<size_t>(ctx->T) * ctx->nu;
    if (u_d < out_d + TN && out_d < u_d + TN)
        return fail(ctx, MPPI_ERR_INVALID_ARG, "u and out must not overlap");
    cudaError_t e = mppi::launch_shift(*ctx, u_d, s, out_d);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "shift launch");
    return MPPI_OK;
}

mppi_status mppi_get_counter(mppi_ctx *ctx, uint64_t *counter) {
    if (!ctx || !counter) return MPPI_ERR_INVALID_ARG;
    unsigned long long v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, ctx->scr.counter, sizeof v, cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "counter read");
    *counter = v;
    return MPPI_OK;
}

mppi_status mppi_set_counter(mppi_ctx *ctx, uint64_t counter) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    cudaError_t e = mppi::launch_store_u64(ctx->scr.counter, counter, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "counter write");
    return MPPI_OK;
}

mppi_status mppi_poll_status(mppi_ctx *ctx) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    unsigned int word = 0;
    cudaError_t e = cudaMemcpyAsync(&word, ctx->scr.status, sizeof word, cudaMemcpyDeviceToHost,
                                    ctx->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(ctx->scr.status, 0, sizeof word, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read");
    for (int code = 1; code < 32; ++code)
        if (word & (1u << code)) {
            ctx->err = code == MPPI_ERR_NUMERIC   ? "every sample cost was non-finite"
                       : code == MPPI_ERR_TIMEOUT ? "a bounded device wait gave up"
                       : code == MPPI_ERR_CHECK   ? "checked mode: a device index was out of range"
                                                  : "device-side error";
            return static_cast<mppi_status>(code);
        }
    return MPPI_OK;
}

const char *mppi_last_error(const mppi_ctx *ctx) { return ctx ? ctx->err.c_str() : ""; }

mppi_status mppi_profile(mppi_ctx *ctx, int enable) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    if (enable) {
        cudaError_t e = cudaStreamSynchronize(ctx->stream);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
        ctx->prof.launches.clear();
        ctx->prof.pool_used = 0;
    }
    ctx->prof.on = enable != 0;
    return MPPI_OK;
}

mppi_status mppi_profile_read(mppi_ctx *ctx, float *ms, int *launches) {
    if (!ctx) return MPPI_ERR_INVALID_ARG;
    cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream synchronize");
    float tot[MPPI_PROF_SLOTS] = {0};
    int cnt[MPPI_PROF_SLOTS] = {0};
    for (const auto &l : ctx->prof.launches) {
        float t = 0.f;
        e = cudaEventElapsedTime(&t, l.second.first, l.second.second);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "event elapsed time");
        if (l.first >= 0 && l.first < MPPI_PROF_SLOTS) {
            tot[l.first] += t;
            cnt[l.first] += 1;
        }
    }
    for (int i = 0; i < MPPI_PROF_SLOTS; ++i) {
        if (ms) ms[i] = tot[i];
        if (launches) launches[i] = cnt[i];
    }
    return MPPI_OK;
}

mppi_status mppi_sample_noise(uint64_t seed, uint64_t step, int K, int Q, uint32_t *bits_d,
                              float *z_d, void *cuda_stream) {
    if (K < 0 || Q < 0 || (!bits_d && !z_d)) return MPPI_ERR_INVALID_ARG;
    if (static_cast<long long>(K) * Q > (1ll << 31) / 4) return MPPI_ERR_INVALID_ARG;
    cudaError_t e = mppi::launch_sample_noise(seed, step, K, Q, bits_d, z_d,
                                              static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? MPPI_OK : MPPI_ERR_CUDA;
}

}  // extern "C"
