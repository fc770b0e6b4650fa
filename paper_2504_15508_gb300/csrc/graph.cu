// A plan's force evaluation captured once as a CUDA graph and replayed.
//
// The step is a fixed sequence of about a dozen kernels and memsets whose
// arguments, apart from the sites, do not change between steps of a run.  The
// graph is captured from one ordinary compute call; on replay, new position
// and charge pointers are patched into the kernel nodes that read them (the
// one-pass site sort and its fallback), so a caller may feed a different
// resident frame every step without copying it.  Outputs (energy, forces, virial), the site count
// and the plan's options are those of the capture.
#include <cstring>
#include <new>
#include <vector>

#include "internal.cuh"
#include "plan.cuh"

using namespace pppm;

struct pppm_graph {
    pppm_plan* plan = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // the kernel nodes that read the sites (arguments (Geo, pos, q, n,
    // DirectArgs) or (Geo, pos, q, n, six pointers)): copies of their
    // parameters, so that new site pointers can be patched into each
    struct SiteNode {
        cudaGraphNode_t node = nullptr;
        cudaKernelNodeParams params{};
        Geo geo{};
        int n = 0;
        bool compact = false;      // the compact layout's binning kernel
        DirectArgs<float> args{};  // the same layout for both precisions (pointers and ints)
        void* ptrs[6] = {};        // the binning kernel's other arguments
    };
    std::vector<SiteNode> sites;
    const void* pos = nullptr;
    const void* q = nullptr;
    int in_size = 4;  // bytes per input value (float or double)
    uint64_t gen = 0;  // plan state at capture
};

namespace {

template <typename In>
int graph_create(pppm_plan* P, void* stream, const In* pos, const In* q, int64_t n, double* energy, In* forces,
                 double* virial, pppm_graph** out) {
    if (!out) return PPPM_ERR_INVALID_ARG;
    *out = nullptr;
    if (!P || n <= 0 || !pos || !q || !energy || !forces || !virial) return PPPM_ERR_INVALID_ARG;
    if (P->prof_on) return PPPM_ERR_INVALID_ARG;  // per-kernel events are not captured
    if (cudaSetDevice(P->device) != cudaSuccess) return PPPM_ERR_CUDA;
    cudaStream_t s = (cudaStream_t)stream;
    if (!s) return PPPM_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
    // one eager call sets up tiles and site buffers (allocations cannot be captured)
    int rc = sizeof(In) == 4 ? pppm_compute_f32(P, stream, (const float*)pos, (const float*)q, n, energy,
                                                (float*)forces, virial)
                             : pppm_compute(P, stream, (const double*)pos, (const double*)q, n, energy,
                                            (double*)forces, virial);
    if (rc != PPPM_OK) return rc;
    pppm_graph* G = new (std::nothrow) pppm_graph();
    if (!G) return PPPM_ERR_CUDA;
    G->plan = P;
    G->in_size = (int)sizeof(In);
    auto fail = [&](int code) {
        pppm_graph_destroy(G);
        return code;
    };
    if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return fail(PPPM_ERR_CUDA);
    rc = sizeof(In) == 4 ? pppm_compute_f32(P, stream, (const float*)pos, (const float*)q, n, energy, (float*)forces,
                                            virial)
                         : pppm_compute(P, stream, (const double*)pos, (const double*)q, n, energy,
                                        (double*)forces, virial);
    cudaGraph_t g = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(s, &g);
    G->graph = g;
    if (rc != PPPM_OK) return fail(rc);
    if (ce != cudaSuccess || !g) return fail(PPPM_ERR_CUDA);
    size_t nn = 0;
    if (cudaGraphGetNodes(g, nullptr, &nn) != cudaSuccess || nn == 0) return fail(PPPM_ERR_CUDA);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(g, nodes.data(), &nn) != cudaSuccess) return fail(PPPM_ERR_CUDA);
    static_assert(sizeof(DirectArgs<float>) == sizeof(DirectArgs<double>), "site-kernel arguments");
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(nd, &t) != cudaSuccess || t != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
        const bool compact = is_bin_kernel(kp.func);
        if (!compact && !is_site_kernel(kp.func)) continue;
        pppm_graph::SiteNode sn;
        sn.node = nd;
        sn.params = kp;
        sn.compact = compact;
        void** a = kp.kernelParams;
        std::memcpy(&sn.geo, a[0], sizeof(Geo));
        std::memcpy(&sn.n, a[3], sizeof(int));
        if (compact)
            for (int k = 0; k < 6; ++k) std::memcpy(&sn.ptrs[k], a[4 + k], sizeof(void*));
        else
            std::memcpy(&sn.args, a[4], sizeof(DirectArgs<float>));
        G->sites.push_back(sn);
    }
    if (G->sites.empty()) return fail(PPPM_ERR_CUDA);  // the step reads its sites somewhere
    G->pos = pos;
    G->q = q;
    if (cudaGraphInstantiate(&G->exec, g, 0) != cudaSuccess) return fail(PPPM_ERR_CUDA);
    G->gen = P->gen;
    *out = G;
    return PPPM_OK;
}

template <typename In>
int graph_launch(pppm_graph* G, void* stream, const In* pos, const In* q) {
    if (!G || !G->exec || (int)sizeof(In) != G->in_size) return PPPM_ERR_INVALID_ARG;
    // the plan reallocated a buffer or changed an option since the capture
    if (G->plan->gen != G->gen) return PPPM_ERR_INVALID_ARG;
    if (cudaSetDevice(G->plan->device) != cudaSuccess) return PPPM_ERR_CUDA;
    const void* np = pos ? (const void*)pos : G->pos;
    const void* nq = q ? (const void*)q : G->q;
    if (np != G->pos || nq != G->q) {
        for (pppm_graph::SiteNode& sn : G->sites) {
            void* args[10] = {&sn.geo, (void*)&np, (void*)&nq, &sn.n, &sn.args};
            if (sn.compact)
                for (int k = 0; k < 6; ++k) args[4 + k] = &sn.ptrs[k];
            cudaKernelNodeParams kp = sn.params;
            kp.kernelParams = args;
            kp.extra = nullptr;
            if (cudaGraphExecKernelNodeSetParams(G->exec, sn.node, &kp) != cudaSuccess) return PPPM_ERR_CUDA;
        }
        G->pos = np;
        G->q = nq;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaGraphLaunch(G->exec, s) != cudaSuccess) return PPPM_ERR_CUDA;
    G->plan->last = s;
    return PPPM_OK;
}

}  // namespace

extern "C" {

int pppm_graph_create(pppm_plan* plan, void* stream, const double* pos, const double* q, int64_t n, double* energy,
                      double* forces, double* virial, pppm_graph** out) {
    return graph_create<double>(plan, stream, pos, q, n, energy, forces, virial, out);
}

int pppm_graph_create_f32(pppm_plan* plan, void* stream, const float* pos, const float* q, int64_t n,
                          double* energy, float* forces, double* virial, pppm_graph** out) {
    return graph_create<float>(plan, stream, pos, q, n, energy, forces, virial, out);
}

int pppm_graph_launch(pppm_graph* graph, void* stream, const double* pos, const double* q) {
    return graph_launch<double>(graph, stream, pos, q);
}

int pppm_graph_launch_f32(pppm_graph* graph, void* stream, const float* pos, const float* q) {
    return graph_launch<float>(graph, stream, pos, q);
}

void pppm_graph_destroy(pppm_graph* graph) {
    if (!graph) return;
    if (graph->plan) cudaSetDevice(graph->plan->device);
    if (graph->exec) cudaGraphExecDestroy(graph->exec);
    if (graph->graph) cudaGraphDestroy(graph->graph);
    delete graph;
}

}  // extern "C"
