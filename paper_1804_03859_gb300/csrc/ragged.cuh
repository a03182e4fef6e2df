// Ragged FP32 stepper: independent solves on grids of different sizes
// advanced by one persistent launch per step kernel (Sec. 3.2's products
// with M for many eigenproblems at once).
//
// Each grid (nx, ny, dt) is a group: a batched FP32 stepper (StepperImpl)
// with one member per solve, which owns the group's fields, spectra,
// operator tables and base-derived fields.  A time step of every group is
// six launches, one per step kernel, each covering the blocks of all groups:
// a block takes items (group, member, block of that member) from a
// grid-stride list, runs the kernel body of the six-kernel step on them and
// returns when the list is done (persistent blocks).  Every group's plan
// keeps the same block size (2^3 elements a thread; sequences per block
// chosen so that sequences x length is the same for every grid), so one
// launch shape serves all grids; the dynamic shared memory is the largest
// group's.  Group descriptors (fields, plan, steps per product) travel in
// the kernel parameters.
//
// Groups differ in their time step, so a product with M (T/dt steps) takes
// a different number of steps per group: a product round runs as many
// steps as the longest group needs, and a group's items are skipped once
// its own steps are done.  The round is captured once as a CUDA graph and
// replayed; which members take part is read from device memory at run
// time, so one graph serves every round.
#pragma once

#include <string>
#include <vector>

namespace nsstab {

struct RagParams {
    int ngroups;
    int step;                                   // step of the round this launch performs
    int first_item[kRagMaxGroups + 1];          // prefix of members x blocks over the groups
    int blocks[kRagMaxGroups];                  // blocks per member of this kernel in group g
    int nsteps[kRagMaxGroups];                  // steps of one product in group g
    int per[kRagMaxGroups], logper[kRagMaxGroups];
    float scale[kRagMaxGroups];                 // 1/(nx ny)
    Fields<float> f[kRagMaxGroups];
};

template <int KID>
__global__ void __launch_bounds__(512) k_ragged(const __grid_constant__ RagParams P, float c1, float c0, bool first) {
    const int total = P.first_item[P.ngroups];
    for (int it = blockIdx.x; it < total; it += gridDim.x) {
        int g = 0;
        while (g + 1 < P.ngroups && it >= P.first_item[g + 1]) ++g;
        if (P.step >= P.nsteps[g]) continue;   // this group's product is done
        const int local = it - P.first_item[g];
        const int m = local / P.blocks[g], bx = local - m * P.blocks[g];
        Fields<float> f = P.f[g];
        if (!member_view_at(f, m)) continue;   // finished solve
        const int per = P.per[g], lp = P.logper[g];
        if constexpr (KID == KCOLP) col_poisson_body<float, 3, true>(f, bx, per, P.scale[g]);
        if constexpr (KID == KINVP) row_inverse_body<float, 3, INV_UV>(f, bx, per, lp);
        if constexpr (KID == KFWDR) row_forward_body<float, FWD_RHS_LIN, 3>(f, bx, per, lp, false, true);
        if constexpr (KID == KCOLU) col_update_body<float, 3>(f, bx, per, c1, c0, first);
        if constexpr (KID == KINVR) row_inverse_body<float, 3, INV_WUV>(f, bx, per, lp);
        if constexpr (KID == KFWDP) row_forward_body<float, FWD_PEN_LIN, 3>(f, bx, per, lp, false, true);
        __syncthreads();   // shared memory is reused by the next item
    }
}

class RaggedF32 : public RaggedBase {
  public:
    explicit RaggedF32(cudaStream_t s) : stream_(s) {}
    ~RaggedF32() override {
        cudaStreamSynchronize(stream_);
        if (graph_) cudaGraphExecDestroy(graph_);
        if (cap_) cudaStreamDestroy(cap_);
        for (auto& g : g_) delete g.st;
    }

    // A group of k solves on one grid: Reynolds numbers and diameters per
    // solve, their base flows (device FP64 [ny][nx] each), nsteps = T/dt.
    int add_group(const nsstab_config& cfg, int k, const double* Re, const double* D, int nsteps,
                  const double* const* bases) override {
        if ((int)g_.size() >= kRagMaxGroups) {
            set_error("ragged stepper: too many grids in one launch");
            return NSSTAB_ERR_INVALID_ARG;
        }
        nsstab_config c = cfg;
        c.precision = 32;
        Group gr;
        gr.st = new StepperImpl<float>(c, k, Re, D, 1, stream_);
        g_.push_back(gr);
        Group& G = g_.back();
        NS_TRY(G.st->init());
        NS_TRY(G.st->set_base_ptrs(bases));
        G.k = k;
        G.nsteps = nsteps;
        G.n = (long)c.nx * c.ny;
        G.mem0 = members_;
        members_ += k;
        return NSSTAB_OK;
    }

    int members() const override { return members_; }
    int groups() const override { return (int)g_.size(); }
    long n_of(int m) const override { return g_[group_of(m)].n; }

    // Plans with one block size per kernel across the groups, and the round
    // of smax steps captured as a graph.
    int finalize() override {
        if (g_.empty()) {
            set_error("ragged stepper: no groups");
            return NSSTAB_ERR_INVALID_ARG;
        }
        int nx_max = 0, ny_max = 0;
        smax_ = 0;
        for (auto& G : g_) {
            nx_max = std::max(nx_max, G.st->nx_);
            ny_max = std::max(ny_max, G.st->ny_);
            smax_ = std::max(smax_, G.nsteps);
        }
        for (int kid = 0; kid < kNumStepKernels; ++kid) {
            const bool row = (kid == KINVP || kid == KFWDR || kid == KINVR || kid == KFWDP);
            // sequences x length per block: aim for 128 (rows) or 64 (columns)
            // threads, fewer where a small grid has too few sequences
            const int nmax = row ? nx_max : ny_max;
            int unit = std::max(nmax, row ? 1024 : 512);
            while (unit > nmax) {
                bool fits = true;
                for (auto& G : g_) {
                    const int N = row ? G.st->nx_ : G.st->ny_;
                    fits = fits && G.st->make_plan(kid, 3, unit / N, 1).ok;
                }
                if (fits) break;
                unit >>= 1;
            }
            RagParams& P = P_[kid];
            std::memset(&P, 0, sizeof(P));
            P.ngroups = (int)g_.size();
            threads_[kid] = 0;
            smem_[kid] = 0;
            for (int gi = 0; gi < (int)g_.size(); ++gi) {
                StepperImpl<float>& S = *g_[gi].st;
                const int N = row ? S.nx_ : S.ny_;
                const int per = unit / N;
                const Launch L = S.make_plan(kid, 3, per, 1);
                if (!L.ok) {
                    set_error("ragged stepper: no common launch shape for grid " + std::to_string(S.nx_) + "x" +
                              std::to_string(S.ny_));
                    return NSSTAB_ERR_INVALID_ARG;
                }
                if (threads_[kid] && L.threads != threads_[kid]) {
                    set_error("ragged stepper: block sizes differ between grids");
                    return NSSTAB_ERR_INVALID_ARG;
                }
                threads_[kid] = L.threads;
                smem_[kid] = std::max(smem_[kid], L.smem);
                P.blocks[gi] = L.blocks;
                P.per[gi] = L.per;
                P.logper[gi] = L.logper;
                P.nsteps[gi] = g_[gi].nsteps;
                P.scale[gi] = S.scale_;
                P.f[gi] = S.f_;
                P.first_item[gi + 1] = P.first_item[gi] + g_[gi].k * L.blocks;
            }
            const int sm = (int)kMaxSmem;
#define NS_RAG_ATTR(K) NS_CUDA(cudaFuncSetAttribute(k_ragged<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm))
            switch (kid) {
                case KCOLP: NS_RAG_ATTR(KCOLP); break;
                case KINVP: NS_RAG_ATTR(KINVP); break;
                case KFWDR: NS_RAG_ATTR(KFWDR); break;
                case KCOLU: NS_RAG_ATTR(KCOLU); break;
                case KINVR: NS_RAG_ATTR(KINVR); break;
                default: NS_RAG_ATTR(KFWDP); break;
            }
#undef NS_RAG_ATTR
            // persistent grid: every item list runs over at most 4 blocks per SM
            blocks_[kid] = std::max(1, std::min(P.first_item[P.ngroups], 4 * 152));
        }
        NS_CUDA(cudaStreamCreateWithFlags(&cap_, cudaStreamNonBlocking));
        cudaGraph_t gph = nullptr;
        NS_CUDA(cudaStreamBeginCapture(cap_, cudaStreamCaptureModeThreadLocal));
        int rc = NSSTAB_OK;
        for (int s = 0; s < smax_ && rc == NSSTAB_OK; ++s) rc = issue_step(cap_, s);
        const cudaError_t ec = cudaStreamEndCapture(cap_, &gph);
        if (rc != NSSTAB_OK) {
            if (gph) cudaGraphDestroy(gph);
            return rc;
        }
        NS_CUDA(ec);
        const cudaError_t ei = cudaGraphInstantiate(&graph_, gph, 0);
        cudaGraphDestroy(gph);
        NS_CUDA(ei);
        return NSSTAB_OK;
    }

    // out[m] = M_m in[m] for every member with a non-null in[m] (global
    // member order: group by group), FP64 device vectors of its grid.
    int product(const double* const* in, double* const* out) override {
        for (auto& G : g_) {
            StepperImpl<float>& S = *G.st;
            std::vector<unsigned char> a(G.k);
            std::vector<const double*> pi(in + G.mem0, in + G.mem0 + G.k);
            bool any = false;
            for (int i = 0; i < G.k; ++i) {
                a[i] = pi[i] != nullptr;
                any = any || a[i];
            }
            NS_TRY(S.set_active(a));
            if (!any) continue;
            NS_TRY(S.gather(pi.data()));
            NS_TRY(S.transform_W());
        }
        NS_CUDA(cudaGraphLaunch(graph_, stream_));
        for (auto& G : g_) {
            std::vector<double*> po(out + G.mem0, out + G.mem0 + G.k);
            bool any = false;
            for (int i = 0; i < G.k; ++i) any = any || (in[G.mem0 + i] != nullptr);
            if (any) NS_TRY(G.st->scatter(G.st->f_.W, po.data()));
        }
        return NSSTAB_OK;
    }

    int launches_per_round() const override { return kNumStepKernels * smax_; }

  private:
    struct Group {
        StepperImpl<float>* st = nullptr;
        int k = 0, nsteps = 0, mem0 = 0;
        long n = 0;
    };
    std::vector<Group> g_;
    cudaStream_t stream_;
    cudaStream_t cap_ = nullptr;
    cudaGraphExec_t graph_ = nullptr;
    int members_ = 0, smax_ = 0;
    RagParams P_[kNumStepKernels];
    int threads_[kNumStepKernels] = {0};
    size_t smem_[kNumStepKernels] = {0};
    int blocks_[kNumStepKernels] = {0};

    int group_of(int m) const {
        int g = 0;
        while (g + 1 < (int)g_.size() && m >= g_[g + 1].mem0) ++g;
        return g;
    }

    int issue_step(cudaStream_t st, int s) {
        const bool first = (s == 0);
        const float c1 = first ? 1.f : 1.5f, c0 = first ? 0.f : -0.5f;
        for (int kid = 0; kid < kNumStepKernels; ++kid) {
            P_[kid].step = s;
            const dim3 grid(blocks_[kid]), blk(threads_[kid]);
            switch (kid) {
                case KCOLP: k_ragged<KCOLP><<<grid, blk, smem_[kid], st>>>(P_[kid], c1, c0, first); break;
                case KINVP: k_ragged<KINVP><<<grid, blk, smem_[kid], st>>>(P_[kid], c1, c0, first); break;
                case KFWDR: k_ragged<KFWDR><<<grid, blk, smem_[kid], st>>>(P_[kid], c1, c0, first); break;
                case KCOLU: k_ragged<KCOLU><<<grid, blk, smem_[kid], st>>>(P_[kid], c1, c0, first); break;
                case KINVR: k_ragged<KINVR><<<grid, blk, smem_[kid], st>>>(P_[kid], c1, c0, first); break;
                default: k_ragged<KFWDP><<<grid, blk, smem_[kid], st>>>(P_[kid], c1, c0, first); break;
            }
            NS_LAUNCH_CHECK();
        }
        return NSSTAB_OK;
    }
};

}  // namespace nsstab
