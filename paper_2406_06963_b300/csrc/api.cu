// C ABI of libdhrs: errors, scenes, tracing entry point and sessions.
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"

namespace dhr {

static thread_local std::string g_error;

dhr_status set_error(dhr_status s, const char* fmt, ...) {
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_error = buf;
    return s;
}

void clear_error() { g_error.clear(); }

static std::vector<DebugReader>& debug_readers() {
    static std::vector<DebugReader> v;
    return v;
}
void debug_register(DebugReader f) { debug_readers().push_back(f); }

#ifdef DHR_DEBUG
// reads element 5 of a one-element buffer through the bounds check, which
// records the event and reads element 0 instead
__global__ void debug_selftest_kernel(const int* buf, int* out) { out[0] = buf[dbg_index(5, 1, kSiteSelfTest)]; }
#endif

dhr_status svgf_create(int32_t w, int32_t h, dhr_precision prec, dhr_svgf_state** out);
void svgf_free(dhr_svgf_state* s);
uint64_t svgf_history_bytes(const dhr_svgf_state* s);
dhr_status svgf_history_copy(dhr_svgf_state* s, void* h, bool to_host, cudaStream_t st);
dhr_status svgf_run(dhr_svgf_state* s, const dhr_gbuffer* cur, const dhr_gbuffer* prev, const dhr_camera* cam,
                    const dhr_camera* cam_prev, const uint8_t* mask, const uint8_t* ao,
                    const dhr_svgf_params* prm, float* ao_out, float* sh_out, cudaStream_t st);
dhr_status check_svgf_params(const dhr_svgf_params* p);

static dhr_status check_camera(const dhr_camera* c) {
    DHR_CHECK_ARG(c, "camera: null");
    DHR_CHECK_ARG(c->width > 0 && c->height > 0 && c->width <= 16384 && c->height <= 16384,
                  "camera: bad size %dx%d", c->width, c->height);
    DHR_CHECK_ARG(c->tan_half_fov_y > 0.0f, "camera: tan_half_fov_y must be > 0");
    return DHR_OK;
}

static dhr_status check_gbuffer(const dhr_gbuffer* g, int w, int h) {
    DHR_CHECK_ARG(g && g->depth_normal && g->mesh_id, "gbuffer: null pointer");
    DHR_CHECK_ARG(g->width == w && g->height == h, "gbuffer: size %dx%d does not match %dx%d", g->width,
                  g->height, w, h);
    DHR_CHECK_ARG(g->precision == DHR_FP32 || g->precision == DHR_FP16, "gbuffer: bad precision");
    DHR_CHECK_ARG(((uintptr_t)g->depth_normal & 15u) == 0, "gbuffer: depth_normal not 16-byte aligned");
    return DHR_OK;
}

}  // namespace dhr

using namespace dhr;

extern "C" const char* dhr_last_error(void) { return g_error.c_str(); }

// ------------------------------------------------------------ debug build
extern "C" dhr_status dhr_debug_status(uint64_t* first_error, int32_t* debug_build) {
    clear_error();
    DHR_CHECK_ARG(first_error && debug_build, "debug_status: null pointer");
    *first_error = 0;
#ifdef DHR_DEBUG
    *debug_build = 1;
    DHR_CUDA_TRY(cudaDeviceSynchronize());   // the kernels whose checks are read have finished
    for (DebugReader f : debug_readers()) {
        const unsigned long long v = f();
        if (v && !*first_error) *first_error = v;
    }
#else
    *debug_build = 0;
#endif
    return DHR_OK;
}

extern "C" dhr_status dhr_debug_selftest(void* stream) {
    clear_error();
#ifdef DHR_DEBUG
    int* buf = nullptr;
    DHR_CUDA_TRY(cudaMalloc((void**)&buf, 2 * sizeof(int)));
    cudaStream_t st = as_stream(stream);
    cudaError_t e = cudaMemsetAsync(buf, 0, 2 * sizeof(int), st);
    if (e == cudaSuccess) {
        debug_selftest_kernel<<<1, 1, 0, st>>>(buf, buf + 1);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(buf);
    if (e != cudaSuccess) return set_error(DHR_ERR_CUDA, "debug_selftest: %s", cudaGetErrorString(e));
    return DHR_OK;
#else
    (void)stream;
    return set_error(DHR_ERR_STATE, "debug_selftest: not a DHR_DEBUG build");
#endif
}

// ------------------------------------------------------------------ scene
extern "C" dhr_status dhr_create_scene(const dhr_scene_desc* desc, void* stream, dhr_scene** out) {
    clear_error();
    DHR_CHECK_ARG(desc && out, "create_scene: null pointer");
    *out = nullptr;
    DHR_CHECK_ARG(desc->n_triangles == 0 || (desc->vertices && desc->indices),
                  "create_scene: null vertex or index array");
    DHR_CHECK_ARG(desc->n_triangles < (1u << 31), "create_scene: too many triangles");
    DHR_CHECK_ARG(desc->builder == DHR_BUILD_PLOC || desc->builder == DHR_BUILD_LBVH, "create_scene: bad builder");
    cudaStream_t st = as_stream(stream);
    auto* sc = new dhr_scene();
    float* v = nullptr;
    uint32_t* idx = nullptr;
    uint32_t* mesh = nullptr;
    dhr_status s = DHR_OK;
    const size_t nv = desc->n_vertices, nt = desc->n_triangles;
    if (nt > 0) {
        cudaError_t e = cudaMalloc(&v, nv * 12 + 16);
        if (!e) e = cudaMalloc(&idx, nt * 12 + 16);
        if (!e && desc->mesh_ids) e = cudaMalloc(&mesh, nt * 4 + 16);
        if (!e) e = cudaMemcpyAsync(v, desc->vertices, nv * 12, cudaMemcpyHostToDevice, st);
        if (!e) e = cudaMemcpyAsync(idx, desc->indices, nt * 12, cudaMemcpyHostToDevice, st);
        if (!e && mesh) e = cudaMemcpyAsync(mesh, desc->mesh_ids, nt * 4, cudaMemcpyHostToDevice, st);
        if (e)
            s = set_error(e == cudaErrorMemoryAllocation ? DHR_ERR_OOM : DHR_ERR_CUDA, "create_scene: %s",
                          cudaGetErrorString(e));
        if (s == DHR_OK) s = build_lbvh(v, idx, mesh, desc->n_vertices, desc->n_triangles, st, sc, desc->builder);
        if (s == DHR_OK) s = build_chunk_boxes(sc, st);
        if (s == DHR_OK) s = build_seed_grid(sc, st);
        cudaStreamSynchronize(st);
    }
    cudaFree(v);
    cudaFree(idx);
    cudaFree(mesh);
    if (s != DHR_OK) {
        dhr_destroy_scene(sc);
        return s;
    }
    *out = sc;
    return DHR_OK;
}

extern "C" void dhr_destroy_scene(dhr_scene* sc) {
    if (!sc) return;
    cudaFree(sc->nodes);
    cudaFree(sc->tris);
    cudaFree(sc->chunk_box);
    cudaFree(const_cast<int4*>(sc->seeds.cells));
    delete sc;
}

extern "C" dhr_status dhr_scene_get_info(const dhr_scene* sc, dhr_scene_info* out) {
    clear_error();
    DHR_CHECK_ARG(sc && out, "scene_get_info: null pointer");
    out->n_triangles = sc->n_tris;
    out->n_nodes = sc->n_nodes;
    out->height = sc->height;
    out->device_bytes = sc->bytes;
    out->build_ms = sc->build_ms;
    return DHR_OK;
}

// ------------------------------------------------------------------ trace
namespace dhr {
dhr_status dhr_trace_visibility_events(const dhr_scene* scene, const dhr_camera* cam, const dhr_trace_params* params,
                                       dhr_gbuffer* gbuf_out, uint8_t* shadow_mask_out, uint8_t* ao_count_out,
                                       cudaStream_t st, cudaEvent_t after_primary) {
    DHR_CHECK_ARG(scene, "trace_visibility: null scene");
    DHR_TRY(check_camera(cam));
    DHR_TRY(check_trace_params(params));
    DHR_TRY(check_gbuffer(gbuf_out, cam->width, cam->height));
    DHR_CHECK_ARG(shadow_mask_out && ao_count_out, "trace_visibility: null output");
    return launch_trace(scene, cam, params, gbuf_out, shadow_mask_out, ao_count_out, st, nullptr, after_primary);
}
}  // namespace dhr

extern "C" dhr_status dhr_trace_visibility(const dhr_scene* scene, const dhr_camera* cam,
                                           const dhr_trace_params* params, dhr_gbuffer* gbuf_out,
                                           uint8_t* shadow_mask_out, uint8_t* ao_count_out, void* stream) {
    clear_error();
    return dhr_trace_visibility_events(scene, cam, params, gbuf_out, shadow_mask_out, ao_count_out,
                                       as_stream(stream), nullptr);
}

extern "C" dhr_status dhr_trace_visibility_selective(const dhr_scene* scene, const dhr_camera* cam,
                                                     const dhr_trace_params* params,
                                                     const dhr_shadow_map* const* maps, dhr_gbuffer* gbuf_out,
                                                     uint8_t* shadow_mask_out, uint8_t* ao_count_out,
                                                     uint8_t* ray_mask_out, void* stream) {
    clear_error();
    DHR_CHECK_ARG(scene, "trace_visibility_selective: null scene");
    DHR_TRY(check_camera(cam));
    DHR_TRY(check_trace_params(params));
    DHR_TRY(check_gbuffer(gbuf_out, cam->width, cam->height));
    DHR_CHECK_ARG(shadow_mask_out && ao_count_out, "trace_visibility_selective: null output");
    return launch_trace_selective(scene, cam, params, maps, gbuf_out, shadow_mask_out, ao_count_out, ray_mask_out,
                                  as_stream(stream));
}

// ---------------------------------------------------------------- session
// Consecutive frames are pipelined: the trace of frame N+1 runs on the
// session's trace stream while the SVGF of frame N runs on its SVGF stream
// (the trace is bound by instruction issue and L1, the filter by latency and
// special-function throughput, so the two overlap well).  G-buffers and raw
// trace outputs rotate through kRing slots; a slot is traced into again only
// after the SVGF of the frame that last read it (as history) has finished.
constexpr int kRing = 3;

struct dhr_session {
    const dhr_scene* scene = nullptr;
    int32_t w = 0, h = 0;
    dhr_precision prec = DHR_FP32;
    dhr_trace_params tp{};
    dhr_svgf_params sp{};
    void* gdn[kRing] = {};
    uint32_t* gmesh[kRing] = {};
    uint8_t* mask[kRing] = {};
    uint8_t* ao[kRing] = {};
    cudaStream_t trace_st = nullptr, svgf_st = nullptr;
    cudaEvent_t traced = nullptr, caller = nullptr;
    cudaEvent_t filtered[kRing] = {};   // SVGF done for the frame traced into that slot
    float* out = nullptr;         // [2][W*H]: filtered AO, filtered shadow
    float* out_b = nullptr;       // second output buffer of the streaming host path
    cudaStream_t copy_st = nullptr;
    cudaEvent_t computed[2] = {nullptr, nullptr}, copied[2] = {nullptr, nullptr};
    cudaEvent_t ticket_done[4] = {};   // copy of ticket t done: ticket_done[(t - 1) % 4]
    uint64_t tickets = 0;         // streaming frames issued
    dhr_svgf_state* svgf = nullptr;
    dhr_camera cam_prev{};
    bool has_prev = false;
    int cur = 0;
};

extern "C" void dhr_session_destroy(dhr_session* s) {
    if (!s) return;
    if (s->trace_st) cudaStreamSynchronize(s->trace_st);
    if (s->svgf_st) cudaStreamSynchronize(s->svgf_st);
    if (s->copy_st) cudaStreamSynchronize(s->copy_st);
    for (int i = 0; i < kRing; ++i) {
        if (s->filtered[i]) cudaEventDestroy(s->filtered[i]);
        cudaFree(s->gdn[i]);
        cudaFree(s->gmesh[i]);
        cudaFree(s->mask[i]);
        cudaFree(s->ao[i]);
    }
    if (s->traced) cudaEventDestroy(s->traced);
    if (s->caller) cudaEventDestroy(s->caller);
    if (s->trace_st) cudaStreamDestroy(s->trace_st);
    if (s->svgf_st) cudaStreamDestroy(s->svgf_st);
    for (int i = 0; i < 2; ++i) {
        if (s->computed[i]) cudaEventDestroy(s->computed[i]);
        if (s->copied[i]) cudaEventDestroy(s->copied[i]);
    }
    for (int i = 0; i < 4; ++i)
        if (s->ticket_done[i]) cudaEventDestroy(s->ticket_done[i]);
    if (s->copy_st) cudaStreamDestroy(s->copy_st);
    cudaFree(s->out_b);
    cudaFree(s->out);
    svgf_free(s->svgf);
    delete s;
}

extern "C" dhr_status dhr_session_create(const dhr_scene* scene, int32_t width, int32_t height,
                                         dhr_precision precision, const dhr_trace_params* trace,
                                         const dhr_svgf_params* svgf, dhr_session** out) {
    clear_error();
    DHR_CHECK_ARG(scene && out, "session_create: null pointer");
    DHR_CHECK_ARG(width > 0 && height > 0 && width <= 16384 && height <= 16384, "session_create: bad size");
    DHR_TRY(check_trace_params(trace));
    DHR_TRY(check_svgf_params(svgf));
    *out = nullptr;
    auto* s = new dhr_session();
    s->scene = scene;
    s->w = width;
    s->h = height;
    s->prec = precision;
    s->tp = *trace;
    s->sp = *svgf;
    const size_t n = (size_t)width * height;
    const size_t gb = precision == DHR_FP16 ? 8 : 16;
    cudaError_t e = cudaSuccess;
    for (int i = 0; i < kRing && !e; ++i) {
        e = cudaMalloc(&s->gdn[i], n * gb);
        if (!e) e = cudaMalloc((void**)&s->gmesh[i], n * 4);
        if (!e) e = cudaMalloc((void**)&s->mask[i], n);
        if (!e) e = cudaMalloc((void**)&s->ao[i], n);
        if (!e) e = cudaEventCreateWithFlags(&s->filtered[i], cudaEventDisableTiming);
    }
    if (!e) e = cudaStreamCreateWithFlags(&s->trace_st, cudaStreamNonBlocking);
    if (!e) e = cudaStreamCreateWithFlags(&s->svgf_st, cudaStreamNonBlocking);
    if (!e) e = cudaEventCreateWithFlags(&s->traced, cudaEventDisableTiming);
    if (!e) e = cudaEventCreateWithFlags(&s->caller, cudaEventDisableTiming);
    if (!e) e = cudaMalloc((void**)&s->out, 2 * n * sizeof(float));
    if (!e) e = cudaMalloc((void**)&s->out_b, 2 * n * sizeof(float));
    if (!e) e = cudaStreamCreateWithFlags(&s->copy_st, cudaStreamNonBlocking);
    for (int i = 0; i < 2 && !e; ++i) {
        e = cudaEventCreateWithFlags(&s->computed[i], cudaEventDisableTiming);
        if (!e) e = cudaEventCreateWithFlags(&s->copied[i], cudaEventDisableTiming);
    }
    for (int i = 0; i < 4 && !e; ++i) e = cudaEventCreateWithFlags(&s->ticket_done[i], cudaEventDisableTiming);
    if (e) {
        cudaGetLastError();
        dhr_session_destroy(s);
        return set_error(e == cudaErrorMemoryAllocation ? DHR_ERR_OOM : DHR_ERR_CUDA, "session_create: %s",
                         cudaGetErrorString(e));
    }
    dhr_status st = svgf_create(width, height, precision, &s->svgf);
    if (st != DHR_OK) {
        dhr_session_destroy(s);
        return st;
    }
    *out = s;
    return DHR_OK;
}

static dhr_gbuffer session_gbuf(const dhr_session* s, int i) {
    dhr_gbuffer g;
    g.precision = s->prec;
    g.width = s->w;
    g.height = s->h;
    g.depth_normal = s->gdn[i];
    g.mesh_id = s->gmesh[i];
    return g;
}

extern "C" dhr_status dhr_step_frame(dhr_session* s, const dhr_camera* cam, uint32_t frame, float* ao_out,
                                     float* shadow_out, void* stream) {
    clear_error();
    DHR_CHECK_ARG(s, "step_frame: null session");
    DHR_TRY(check_camera(cam));
    DHR_CHECK_ARG(cam->width == s->w && cam->height == s->h, "step_frame: camera size %dx%d, session %dx%d",
                  cam->width, cam->height, s->w, s->h);
    cudaStream_t st = as_stream(stream);
    const int b = (s->cur + 1) % kRing;     // this frame's slot; s->cur holds the previous frame
    dhr_gbuffer g = session_gbuf(s, b);
    dhr_gbuffer gp = session_gbuf(s, s->cur);
    dhr_trace_params tp = s->tp;
    tp.frame = frame;
    // slot b was last read (as history) by the SVGF of the frame two steps back
    DHR_CUDA_TRY(cudaStreamWaitEvent(s->trace_st, s->filtered[(b + 1) % kRing], 0));
    DHR_TRY(launch_trace(s->scene, cam, &tp, &g, s->mask[b], s->ao[b], s->trace_st));
    DHR_CUDA_TRY(cudaEventRecord(s->traced, s->trace_st));
    const size_t n = (size_t)s->w * s->h;
    float* ao = ao_out ? ao_out : s->out;
    float* sh = shadow_out ? shadow_out : s->out + n;
    // the session's own output buffer may still be read by a streaming copy
    if (!ao_out || !shadow_out) DHR_CUDA_TRY(cudaStreamWaitEvent(st, s->copied[0], 0));
    // the filter writes caller memory: after the caller's earlier work on `stream`
    DHR_CUDA_TRY(cudaEventRecord(s->caller, st));
    DHR_CUDA_TRY(cudaStreamWaitEvent(s->svgf_st, s->caller, 0));
    DHR_CUDA_TRY(cudaStreamWaitEvent(s->svgf_st, s->traced, 0));
    DHR_TRY(svgf_run(s->svgf, &g, s->has_prev ? &gp : nullptr, cam, s->has_prev ? &s->cam_prev : nullptr,
                     s->mask[b], s->ao[b], &s->sp, ao, sh, s->svgf_st));
    DHR_CUDA_TRY(cudaEventRecord(s->filtered[b], s->svgf_st));
    DHR_CUDA_TRY(cudaStreamWaitEvent(st, s->filtered[b], 0));   // results in `stream` order
    s->cur = b;
    s->cam_prev = *cam;
    s->has_prev = true;
    return DHR_OK;
}

extern "C" dhr_status dhr_step_frame_host(dhr_session* s, const dhr_camera* cam, uint32_t frame, float* ao_host,
                                          float* shadow_host, void* stream) {
    DHR_CHECK_ARG(ao_host && shadow_host, "step_frame_host: null output");
    DHR_TRY(dhr_step_frame(s, cam, frame, nullptr, nullptr, stream));
    cudaStream_t st = as_stream(stream);
    const size_t n = (size_t)s->w * s->h;
    DHR_CUDA_TRY(cudaMemcpyAsync(ao_host, s->out, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    DHR_CUDA_TRY(cudaMemcpyAsync(shadow_host, s->out + n, n * sizeof(float), cudaMemcpyDeviceToHost, st));
    DHR_CUDA_TRY(cudaStreamSynchronize(st));
    return DHR_OK;
}

extern "C" dhr_status dhr_step_frame_host_async(dhr_session* s, const dhr_camera* cam, uint32_t frame,
                                                float* ao_host, float* shadow_host, void* stream,
                                                uint64_t* out_ticket) {
    DHR_CHECK_ARG(s && ao_host && shadow_host && out_ticket, "step_frame_host_async: null pointer");
    cudaStream_t st = as_stream(stream);
    const size_t n = (size_t)s->w * s->h;
    const int slot = (int)(s->tickets & 1);
    float* dev = slot ? s->out_b : s->out;
    // the copy of the frame that last used this output buffer reads it: wait on the device
    DHR_CUDA_TRY(cudaStreamWaitEvent(st, s->copied[slot], 0));
    DHR_TRY(dhr_step_frame(s, cam, frame, dev, dev + n, stream));
    DHR_CUDA_TRY(cudaEventRecord(s->computed[slot], st));
    DHR_CUDA_TRY(cudaStreamWaitEvent(s->copy_st, s->computed[slot], 0));
    DHR_CUDA_TRY(cudaMemcpyAsync(ao_host, dev, n * sizeof(float), cudaMemcpyDeviceToHost, s->copy_st));
    DHR_CUDA_TRY(cudaMemcpyAsync(shadow_host, dev + n, n * sizeof(float), cudaMemcpyDeviceToHost, s->copy_st));
    DHR_CUDA_TRY(cudaEventRecord(s->copied[slot], s->copy_st));
    DHR_CUDA_TRY(cudaEventRecord(s->ticket_done[s->tickets % 4], s->copy_st));
    *out_ticket = ++s->tickets;
    return DHR_OK;
}

extern "C" dhr_status dhr_session_wait(dhr_session* s, uint64_t ticket) {
    clear_error();
    DHR_CHECK_ARG(s, "session_wait: null session");
    DHR_CHECK_ARG(ticket >= 1 && ticket <= s->tickets, "session_wait: ticket %llu not issued (last %llu)",
                  (unsigned long long)ticket, (unsigned long long)s->tickets);
    // the event of ticket t, or (after 4 more tickets reused it) of a later
    // copy on the same stream, which completes after t's
    DHR_CUDA_TRY(cudaEventSynchronize(s->ticket_done[(ticket - 1) % 4]));
    return DHR_OK;
}

extern "C" dhr_status dhr_session_get_frame(dhr_session* s, dhr_gbuffer* gbuf, uint8_t** shadow_mask,
                                            uint8_t** ao_count) {
    clear_error();
    DHR_CHECK_ARG(s, "session_get_frame: null session");
    if (gbuf) *gbuf = session_gbuf(s, s->cur);
    if (shadow_mask) *shadow_mask = s->mask[s->cur];
    if (ao_count) *ao_count = s->ao[s->cur];
    return DHR_OK;
}

// ------------------------------------------------------- checkpoint / resume
// Header of a session checkpoint; the buffers follow it: the current
// G-buffer (depth_normal, then mesh ids) and the SVGF history (colour
// history, moments, history lengths).
struct CheckpointHeader {
    uint32_t magic, version;
    int32_t width, height;
    int32_t precision, has_prev;
    dhr_camera cam_prev;
    uint64_t bytes;          // the whole checkpoint, header included
};
constexpr uint32_t kCheckpointMagic = 0x43524844u;   // "DHRC"

static uint64_t checkpoint_bytes(const dhr_session* s) {
    const uint64_t n = (uint64_t)s->w * s->h;
    return sizeof(CheckpointHeader) + n * ((s->prec == DHR_FP16 ? 8 : 16) + 4) + svgf_history_bytes(s->svgf);
}

extern "C" uint64_t dhr_session_checkpoint_bytes(const dhr_session* s) { return s ? checkpoint_bytes(s) : 0; }

extern "C" dhr_status dhr_session_export(dhr_session* s, void* dst, uint64_t size, void* stream) {
    clear_error();
    DHR_CHECK_ARG(s && dst, "session_export: null pointer");
    const uint64_t need = checkpoint_bytes(s);
    DHR_CHECK_ARG(size >= need, "session_export: %llu bytes given, %llu needed", (unsigned long long)size,
                  (unsigned long long)need);
    cudaStream_t st = as_stream(stream);
    // the last frame's filter (which follows its trace) has written the history
    DHR_CUDA_TRY(cudaStreamWaitEvent(st, s->filtered[s->cur], 0));
    CheckpointHeader hd{};
    hd.magic = kCheckpointMagic;
    hd.version = 1;
    hd.width = s->w;
    hd.height = s->h;
    hd.precision = (int32_t)s->prec;
    hd.has_prev = s->has_prev ? 1 : 0;
    hd.cam_prev = s->cam_prev;
    hd.bytes = need;
    memcpy(dst, &hd, sizeof(hd));
    char* p = static_cast<char*>(dst) + sizeof(hd);
    const size_t n = (size_t)s->w * s->h, gb = s->prec == DHR_FP16 ? 8 : 16;
    DHR_CUDA_TRY(cudaMemcpyAsync(p, s->gdn[s->cur], n * gb, cudaMemcpyDeviceToHost, st));
    p += n * gb;
    DHR_CUDA_TRY(cudaMemcpyAsync(p, s->gmesh[s->cur], n * 4, cudaMemcpyDeviceToHost, st));
    p += n * 4;
    DHR_TRY(svgf_history_copy(s->svgf, p, true, st));
    DHR_CUDA_TRY(cudaStreamSynchronize(st));
    return DHR_OK;
}

extern "C" dhr_status dhr_session_import(dhr_session* s, const void* src, uint64_t size, void* stream) {
    clear_error();
    DHR_CHECK_ARG(s && src, "session_import: null pointer");
    DHR_CHECK_ARG(size >= sizeof(CheckpointHeader), "session_import: %llu bytes is no checkpoint",
                  (unsigned long long)size);
    CheckpointHeader hd;
    memcpy(&hd, src, sizeof(hd));
    DHR_CHECK_ARG(hd.magic == kCheckpointMagic && hd.version == 1, "session_import: not a session checkpoint");
    DHR_CHECK_ARG(hd.width == s->w && hd.height == s->h && hd.precision == (int32_t)s->prec,
                  "session_import: checkpoint of a %dx%d session (precision %d), this one is %dx%d (%d)",
                  hd.width, hd.height, hd.precision, s->w, s->h, (int)s->prec);
    const uint64_t need = checkpoint_bytes(s);
    DHR_CHECK_ARG(hd.bytes == need && size >= need, "session_import: checkpoint of %llu bytes, %llu expected",
                  (unsigned long long)hd.bytes, (unsigned long long)need);
    cudaStream_t st = as_stream(stream);
    // nothing of the session may still read or write the buffers
    DHR_CUDA_TRY(cudaStreamSynchronize(s->trace_st));
    DHR_CUDA_TRY(cudaStreamSynchronize(s->svgf_st));
    DHR_CUDA_TRY(cudaStreamSynchronize(s->copy_st));
    const char* p = static_cast<const char*>(src) + sizeof(hd);
    const size_t n = (size_t)s->w * s->h, gb = s->prec == DHR_FP16 ? 8 : 16;
    DHR_CUDA_TRY(cudaMemcpyAsync(s->gdn[s->cur], p, n * gb, cudaMemcpyHostToDevice, st));
    p += n * gb;
    DHR_CUDA_TRY(cudaMemcpyAsync(s->gmesh[s->cur], p, n * 4, cudaMemcpyHostToDevice, st));
    p += n * 4;
    DHR_TRY(svgf_history_copy(s->svgf, const_cast<char*>(p), false, st));
    DHR_CUDA_TRY(cudaStreamSynchronize(st));
    s->cam_prev = hd.cam_prev;
    s->has_prev = hd.has_prev != 0;
    return DHR_OK;
}

extern "C" dhr_status dhr_session_reset(dhr_session* s) {
    clear_error();
    DHR_CHECK_ARG(s, "session_reset: null session");
    s->has_prev = false;
    return DHR_OK;
}
