// Step-graph helpers: one refinement step captured as a CUDA graph whose
// backward branch (Algorithm 1, "if g = 1: backward; optimizer step") is an IF
// conditional node that skipgs_gate_decide sets on the device.  Built with
// stream capture plus cudaStreamBeginCaptureToGraph for the IF body.
#include <new>

#include "common.cuh"

using namespace gsr;

struct gs_graph_s {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    int64_t kernels_main;  // kernel nodes outside conditional bodies
    int64_t kernels_body;  // kernel nodes inside IF bodies
};

namespace {

// IF bodies created by gs_graph_if_begin while a capture is open on this thread.
thread_local cudaGraph_t t_bodies[8];
thread_local int t_n_bodies = 0;

int64_t count_kernel_nodes(cudaGraph_t g) {
    size_t n = 0;
    if (cudaGraphGetNodes(g, nullptr, &n) != cudaSuccess || n == 0) return 0;
    cudaGraphNode_t *nodes = new (std::nothrow) cudaGraphNode_t[n];
    if (!nodes) return -1;
    int64_t k = 0;
    if (cudaGraphGetNodes(g, nodes, &n) == cudaSuccess) {
        for (size_t i = 0; i < n; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++k;
        }
    }
    delete[] nodes;
    return k;
}

__global__ void select_views_kernel(const int32_t *seq, int64_t seq_len, int64_t *iter, int n, int32_t *view_ids,
                                    const gs_camera *pose_src, gs_camera *slots, int tile) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const int64_t it = *iter;
    int64_t next_tile = slots ? slots[0].tile_offset : 0;  // compact layout: from the first slot's offset
    for (int k = 0; k < n; ++k) {
        const int64_t idx = (it * n + k) % seq_len;
        const int32_t vid = seq[idx];
        view_ids[k] = vid;
        if (pose_src && slots) {  // the pose, intrinsics and size; the slot keeps its tile and pixel offsets
            const gs_camera &src = pose_src[vid];
            gs_camera &dst = slots[k];
            for (int a = 0; a < 9; ++a) dst.R[a] = src.R[a];
            for (int a = 0; a < 3; ++a) dst.t[a] = src.t[a];
            dst.fx = src.fx;
            dst.fy = src.fy;
            dst.cx = src.cx;
            dst.cy = src.cy;
            dst.width = src.width;
            dst.height = src.height;
            dst.znear = src.znear;
            if (tile > 0) {  // each view its own tile grid, packed after the previous slot's
                dst.tile_offset = (int32_t)next_tile;
                next_tile += (int64_t)((src.width + tile - 1) / tile) * ((src.height + tile - 1) / tile);
            }
        }
    }
    *iter = it + 1;
}

// Per-view optimizer steps of a batched iteration: gates[k][j] = (j == k) and
// view k opened (or all_open), do_steps[k] = view k opened (or all_open).
__global__ void view_steps_kernel(const uint8_t *g, int n, int all_open, uint8_t *gates, int32_t *do_steps) {
    for (int i = threadIdx.x; i < n * n; i += blockDim.x) {
        const int k = i / n, j = i % n;
        const int open = all_open || (g && g[k]);
        gates[i] = (uint8_t)(j == k && open);
        if (j == 0) do_steps[k] = open;
    }
}

__global__ void log_step_kernel(const int64_t *iter, int n, const float *loss, const uint8_t *g, double *norms2,
                                float *loss_log, uint8_t *g_log, double *norm_log, int64_t cap) {
    const int64_t it = *iter - 1;
    const int64_t k = ((it % cap) + cap) % cap;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        loss_log[k * n + j] = loss[j];
        g_log[k * n + j] = g[j];
    }
    if (threadIdx.x == 0 && norms2 && norm_log) {
        norm_log[2 * k] = norms2[0];
        norm_log[2 * k + 1] = norms2[1];
        norms2[0] = 0.0;
        norms2[1] = 0.0;
    }
}

}  // namespace

extern "C" {

gs_status gs_view_steps(const uint8_t *g, int32_t n, int32_t all_open, uint8_t *gates, int32_t *do_steps,
                        cudaStream_t stream) {
    if (n <= 0 || n > 1024 || !gates || !do_steps || (!g && !all_open)) return GS_ERR_INVALID_ARG;
    view_steps_kernel<<<1, 256, 0, stream>>>(g, n, all_open ? 1 : 0, gates, do_steps);
    GS_TRY_LAUNCH();
    return GS_OK;
}

gs_status gs_log_step(const int64_t *iter, int32_t n, const float *loss, const uint8_t *g, double *norms2,
                      float *loss_log, uint8_t *g_log, double *norm_log, int64_t cap, cudaStream_t stream) {
    if (!iter || n <= 0 || !loss || !g || !loss_log || !g_log || cap <= 0) return GS_ERR_INVALID_ARG;
    log_step_kernel<<<1, 32, 0, stream>>>(iter, n, loss, g, norms2, loss_log, g_log, norm_log, cap);
    GS_TRY_LAUNCH();
    return GS_OK;
}

gs_status gs_graph_begin(cudaStream_t stream) {
    if (!stream) return GS_ERR_INVALID_ARG;  // the legacy default stream cannot be captured
    t_n_bodies = 0;
    GS_TRY(cudaStreamBeginCapture(stream, cudaStreamCaptureModeRelaxed));
    return GS_OK;
}

gs_status gs_graph_cond_create(cudaStream_t stream, cudaGraphConditionalHandle *out) {
    if (!stream || !out) return GS_ERR_INVALID_ARG;
    cudaStreamCaptureStatus status;
    cudaGraph_t graph;
    GS_TRY(cudaStreamGetCaptureInfo(stream, &status, nullptr, &graph, nullptr, nullptr, nullptr));
    if (status != cudaStreamCaptureStatusActive) return GS_ERR_INVALID_ARG;
    GS_TRY(cudaGraphConditionalHandleCreate(out, graph, 0, cudaGraphCondAssignDefault));
    return GS_OK;
}

gs_status gs_graph_if_begin(cudaStream_t stream, cudaGraphConditionalHandle cond, cudaStream_t body_stream) {
    if (!stream || !body_stream || stream == body_stream) return GS_ERR_INVALID_ARG;
    cudaStreamCaptureStatus status;
    cudaGraph_t graph;
    const cudaGraphNode_t *deps = nullptr;
    const cudaGraphEdgeData *edata = nullptr;
    size_t ndeps = 0;
    GS_TRY(cudaStreamGetCaptureInfo(stream, &status, nullptr, &graph, &deps, &edata, &ndeps));
    if (status != cudaStreamCaptureStatusActive) return GS_ERR_INVALID_ARG;
    cudaGraphNodeParams params = {};
    params.type = cudaGraphNodeTypeConditional;
    params.conditional.handle = cond;
    params.conditional.type = cudaGraphCondTypeIf;
    params.conditional.size = 1;
    cudaGraphNode_t node;
    GS_TRY(cudaGraphAddNode(&node, graph, deps, edata, ndeps, &params));
    GS_TRY(cudaStreamUpdateCaptureDependencies(stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaGraph_t body = params.conditional.phGraph_out[0];
    if (t_n_bodies < 8) t_bodies[t_n_bodies++] = body;
    GS_TRY(cudaStreamBeginCaptureToGraph(body_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    return GS_OK;
}

gs_status gs_graph_if_end(cudaStream_t stream, cudaStream_t body_stream) {
    if (!stream || !body_stream) return GS_ERR_INVALID_ARG;
    cudaGraph_t body;
    GS_TRY(cudaStreamEndCapture(body_stream, &body));
    return GS_OK;
}

gs_status gs_graph_end(cudaStream_t stream, gs_graph *out) {
    if (!stream || !out) return GS_ERR_INVALID_ARG;
    cudaGraph_t graph;
    GS_TRY(cudaStreamEndCapture(stream, &graph));
    cudaGraphExec_t exec;
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
        cudaGraphDestroy(graph);
        return GS_ERR_CUDA;
    }
    int64_t kb = 0;
    for (int i = 0; i < t_n_bodies; ++i) kb += count_kernel_nodes(t_bodies[i]);
    t_n_bodies = 0;
    gs_graph_s *g = new (std::nothrow) gs_graph_s{graph, exec, count_kernel_nodes(graph), kb};
    if (!g) {
        cudaGraphExecDestroy(exec);
        cudaGraphDestroy(graph);
        return GS_ERR_CUDA;
    }
    *out = g;
    return GS_OK;
}

gs_status gs_graph_kernel_counts(gs_graph graph, int64_t *out2) {
    if (!graph || !out2) return GS_ERR_INVALID_ARG;
    out2[0] = graph->kernels_main;
    out2[1] = graph->kernels_body;
    return GS_OK;
}

gs_status gs_graph_launch(gs_graph graph, cudaStream_t stream) {
    if (!graph) return GS_ERR_INVALID_ARG;
    GS_TRY(cudaGraphLaunch(graph->exec, stream));
    return GS_OK;
}

gs_status gs_graph_destroy(gs_graph graph) {
    if (!graph) return GS_ERR_INVALID_ARG;
    cudaGraphExecDestroy(graph->exec);
    cudaGraphDestroy(graph->graph);
    delete graph;
    return GS_OK;
}

gs_status gs_select_views(const int32_t *seq, int64_t seq_len, int64_t *iter, int32_t n, int32_t *view_ids,
                          const gs_camera *pose_src, gs_camera *slots, int32_t tile, cudaStream_t stream) {
    if (!seq || seq_len <= 0 || !iter || n <= 0 || !view_ids) return GS_ERR_INVALID_ARG;
    if (tile != 0 && tile != 8 && tile != 16 && tile != 32) return GS_ERR_INVALID_ARG;
    select_views_kernel<<<1, 32, 0, stream>>>(seq, seq_len, iter, n, view_ids, pose_src, slots, tile);
    GS_TRY_LAUNCH();
    return GS_OK;
}

}  // extern "C"
