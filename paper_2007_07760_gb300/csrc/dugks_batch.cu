// dugks_batch.cu -- many independent grids per launch (declared in include/dugks.h).
//
// Host side of the batch: per-grid device memory and descriptors (BatchGrid,
// with TMA tensor maps), the work list of tiles, the per-step launches and
// their CUDA-graph replay. The arithmetic is the fast kernel's, unchanged.
//
// Nothing on the path of a running batch waits for the device: grid memory comes
// from a stream-ordered pool of the batch's own and goes back to it in stream
// order, descriptors and initial fields are uploaded from pinned staging buffers,
// results are read out into pinned buffers, and every host buffer or graph that
// the stream may still use is released only once a fence (an event recorded on
// the stream, numbered in order) shows the stream has passed it. So a server can
// add, retire and collect grids while steps are in flight.
#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/dugks.h"
#include "dugks_host.h"
#include "dugks_internal.h"

using namespace dugks;
using namespace dugks::host;

namespace {

struct Slot {
    bool used = false;
    bool retiring = false;   // read-out enqueued (dugks_batch_retire), result not yet collected
    int nx = 0, ny = 0, pitch = 0, tiles_x = 0, tiles_y = 0;
    size_t plane = 0;
    void *X[2] = {nullptr, nullptr};
    void *phi[3] = {nullptr, nullptr, nullptr};
    int64_t step = 0, target = -1;
    int vel_kind = DUGKS_VEL_UNIFORM;
    double vel[3] = {0, 0, 0};
    bool mass_known = false;
    uint64_t ticket = 0;            // fence after the read-out
    void *pinned = nullptr;         // host buffer the read-out lands in
    size_t pinned_bytes = 0;
    std::vector<unsigned char> desc;   // encoded descriptor (tensor maps); empty: encode at the next rebuild
};

constexpr int GRAPH_STEPS = 8;
// pinned host buffers kept for reuse beyond this are given back
constexpr size_t PINNED_KEEP = (size_t)1 << 30;

}  // namespace

struct dugks_batch {
    dugks_params p{};
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    size_t tsize = 4, ssize = 4;
    int nphi = 2;
    // 8 warps x 3 rows per thread; FP32: 10 x 4 (measured fastest on mixed batches)
    int variant = 4;
    int ctas = 0;
    int ctas_req = 0;   // 0: resident CTAs (grid-stride); < 0: one CTA per tile; > 0: at most that many
    std::vector<Slot> slots;
    cudaMemPool_t pool = nullptr;   // grid memory, descriptors and the work list
    // device side
    void *d_grids = nullptr;
    int grids_cap = 0;
    int4 *d_items = nullptr;
    int items_cap = 0, nitems = 0;
    double *d_partials = nullptr;
    double *d_mass = nullptr;
    int *d_status = nullptr;
    void *d_tmp = nullptr;       // phi read-out / generic mass partials of the waiting calls
    size_t tmp_bytes = 0;
    bool dirty = true;
    cudaGraphExec_t graph = nullptr;
    std::vector<unsigned char> coefs, uniform;
    // fences: events recorded on the stream with increasing tickets
    std::deque<std::pair<uint64_t, cudaEvent_t>> fences;
    std::vector<cudaEvent_t> spare_events;
    uint64_t next_ticket = 1, reached = 0;
    // pinned host buffers free for reuse (by size), and those waiting for a fence
    std::multimap<size_t, void *> pinned_free;
    size_t pinned_free_bytes = 0;
    std::vector<std::tuple<uint64_t, void *, size_t>> pinned_later;
    std::vector<std::pair<uint64_t, cudaGraphExec_t>> graphs_later;
    int sticky = DUGKS_OK;
    std::string err;
};

namespace {

int bfail(dugks_batch *b, int code, const std::string &msg) {
    if (b) {
        if (b->sticky == DUGKS_OK) b->sticky = code;
        b->err = msg;
    }
    return code;
}
int bcuda(dugks_batch *b, cudaError_t e, const char *where) {
    return bfail(b, DUGKS_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

bool fp64(const dugks_batch *b) { return b->p.precision == DUGKS_FP64; }

// ---- stream-ordered device memory ------------------------------------------
cudaError_t pool_alloc(dugks_batch *b, void **p, size_t bytes) {
    cudaError_t e = dev_malloc_pool(p, bytes, b->pool, b->stream);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
    }
    return e;
}
template <typename P>
cudaError_t pool_alloc(dugks_batch *b, P **p, size_t bytes) {
    return pool_alloc(b, reinterpret_cast<void **>(p), bytes);
}
// freed once the work queued on the stream before it has run
void pool_free(dugks_batch *b, void *p) {
    if (p) cudaFreeAsync(p, b->stream);
}

// ---- fences -----------------------------------------------------------------
void consume_not_ready() {
    if (cudaPeekAtLastError() == cudaErrorNotReady) cudaGetLastError();
}

int fence(dugks_batch *b, uint64_t *ticket) {
    cudaEvent_t ev = nullptr;
    if (!b->spare_events.empty()) {
        ev = b->spare_events.back();
        b->spare_events.pop_back();
    } else {
        cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) return bcuda(b, e, "fence event");
    }
    cudaError_t e = cudaEventRecord(ev, b->stream);
    if (e != cudaSuccess) {
        b->spare_events.push_back(ev);
        return bcuda(b, e, "fence record");
    }
    *ticket = b->next_ticket++;
    b->fences.emplace_back(*ticket, ev);
    return DUGKS_OK;
}

void pinned_put(dugks_batch *b, void *p, size_t bytes) {
    if (!p) return;
    b->pinned_free.emplace(bytes, p);
    b->pinned_free_bytes += bytes;
    while (b->pinned_free_bytes > PINNED_KEEP && !b->pinned_free.empty()) {
        auto it = std::prev(b->pinned_free.end());   // the largest goes first
        b->pinned_free_bytes -= it->first;
        cudaFreeHost(it->second);
        b->pinned_free.erase(it);
    }
}

// a pinned buffer of at least `bytes` (reused when one of at most twice the size is free)
int pinned_get(dugks_batch *b, size_t bytes, void **p, size_t *got) {
    bytes = std::max<size_t>(bytes, 256);
    auto it = b->pinned_free.lower_bound(bytes);
    if (it != b->pinned_free.end() && it->first <= 2 * bytes) {
        *p = it->second;
        *got = it->first;
        b->pinned_free_bytes -= it->first;
        b->pinned_free.erase(it);
        return DUGKS_OK;
    }
    if (cudaMallocHost(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return DUGKS_ENOMEM;
    }
    *got = bytes;
    return DUGKS_OK;
}

// gives `p` back once the stream has passed fence `ticket`
void pinned_later(dugks_batch *b, void *p, size_t bytes, uint64_t ticket) {
    if (p) b->pinned_later.emplace_back(ticket, p, bytes);
}

// moves b->reached over every fence the stream has passed and releases what
// waited for them
int advance(dugks_batch *b) {
    int r = DUGKS_OK;
    while (!b->fences.empty()) {
        cudaError_t e = cudaEventQuery(b->fences.front().second);
        if (e == cudaErrorNotReady) {
            consume_not_ready();
            break;
        }
        if (e != cudaSuccess) {
            r = bcuda(b, e, "batch fence");
            break;
        }
        b->reached = b->fences.front().first;
        b->spare_events.push_back(b->fences.front().second);
        b->fences.pop_front();
    }
    auto &pl = b->pinned_later;
    for (size_t i = 0; i < pl.size();) {
        if (std::get<0>(pl[i]) <= b->reached) {
            pinned_put(b, std::get<1>(pl[i]), std::get<2>(pl[i]));
            pl[i] = pl.back();
            pl.pop_back();
        } else {
            i++;
        }
    }
    auto &gl = b->graphs_later;
    for (size_t i = 0; i < gl.size();) {
        if (gl[i].first <= b->reached) {
            cudaGraphExecDestroy(gl[i].second);
            gl[i] = gl.back();
            gl.pop_back();
        } else {
            i++;
        }
    }
    return r;
}

// blocks until the stream has passed fence `ticket`
int wait_ticket(dugks_batch *b, uint64_t ticket) {
    for (auto &f : b->fences)
        if (f.first >= ticket) {
            cudaError_t e = cudaEventSynchronize(f.second);
            if (e != cudaSuccess) return bcuda(b, e, "batch fence wait");
            break;
        }
    return advance(b);
}


size_t plane_of(int nx, int ny, int *pitch_out) {
    const int pitch = (nx + 2 * GHOST + 31) / 32 * 32;
    if (pitch_out) *pitch_out = pitch;
    return (size_t)(ny + 2 * GHOST) * pitch;
}

template <typename T, typename ST>
FastGeom geom(const dugks_batch *b) { return Launch<T, ST>::fast_geom(b->variant); }

FastGeom batch_geom(const dugks_batch *b) {
    switch (b->p.precision) {
    case DUGKS_FP64: return geom<double, double>(b);
    case DUGKS_FP32: return geom<float, float>(b);
    default: return geom<float, __half>(b);
    }
}

int resident_ctas(dugks_batch *b) {
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->dev);
    int per = 1;
    switch (b->p.precision) {
    case DUGKS_FP64: per = Launch<double, double>::batch_ctas_per_sm(b->p.order, b->p.flux, b->variant); break;
    case DUGKS_FP32: per = Launch<float, float>::batch_ctas_per_sm(b->p.order, b->p.flux, b->variant); break;
    default: per = Launch<float, __half>::batch_ctas_per_sm(b->p.order, b->p.flux, b->variant); break;
    }
    return std::max(1, sms) * std::max(1, per);
}

template <typename T>
void fill_uniform(dugks_batch *b, const FastGeom &g) {
    BatchUniform<T> u;
    std::memset(&u, 0, sizeof u);
    const double dt = b->p.cfl, tau = 3.0 * b->p.M, h = 0.5 * dt;
    const double bb = (dt + h) / (2.0 * tau + dt);   // bar f^+ = X + b (g - X)
    u.b = (T)bb;
    u.h = (T)h;
    u.c1 = (T)(2.0 * tau / (2.0 * tau + h));
    u.c2 = (T)(h / (2.0 * tau + h));
    u.c3 = (T)(tau * h / (2.0 * tau + h));
    u.be1 = (T)(4.0 / 3.0 * bb);
    u.ga1 = (T)dt;
    u.tau = (T)tau;
    u.theta_c = (T)(-4.0 / (b->p.W * (b->p.phiA - b->p.phiB)));
    u.phiA = (T)b->p.phiA;
    u.phiB = (T)b->p.phiB;
    u.inv_dt = (T)(1.0 / dt);
    u.qscale = (T)256.0;
    u.qinv = (T)(1.0 / 256.0);
    u.dt = dt;
    u.dtphiu = b->p.dtphiu;
    u.tile_w = g.tile_w;
    u.tile_h = g.tile_h;
    u.status = b->d_status;
    b->uniform.assign(reinterpret_cast<unsigned char *>(&u), reinterpret_cast<unsigned char *>(&u) + sizeof u);
    FaceCoefs<T> cf = make_face_coefs<T>(b->p.order, b->p.flux, h);
    b->coefs.assign(reinterpret_cast<unsigned char *>(&cf), reinterpret_cast<unsigned char *>(&cf) + sizeof cf);
}

// the current graph is destroyed once the stream has passed its launches
void drop_graph(dugks_batch *b) {
    if (!b->graph) return;
    uint64_t t = 0;
    if (fence(b, &t) == DUGKS_OK) {
        b->graphs_later.emplace_back(t, b->graph);
    } else {
        cudaStreamSynchronize(b->stream);
        cudaGraphExecDestroy(b->graph);
    }
    b->graph = nullptr;
}

// Descriptors and work list of all grids, uploaded in stream order from pinned
// staging (the steps already queued keep the old ones). Grids that reached their
// target, or are retiring, keep a frozen descriptor and contribute no tiles.
template <typename T, typename ST>
int rebuild_t(dugks_batch *b) {
    drop_graph(b);
    const FastGeom g = Launch<T, ST>::fast_geom(b->variant);
    const int n = (int)b->slots.size();
    if (n > b->grids_cap) {
        const int cap = std::max(16, n * 2);
        void *grids = nullptr;
        double *mass = nullptr;
        if (pool_alloc(b, &grids, (size_t)cap * sizeof(BatchGrid<T>)) != cudaSuccess ||
            pool_alloc(b, &mass, (size_t)cap * sizeof(double)) != cudaSuccess) {
            pool_free(b, grids);
            return bfail(b, DUGKS_ENOMEM, "batch descriptors");
        }
        cudaMemsetAsync(mass, 0, (size_t)cap * sizeof(double), b->stream);
        if (b->d_mass)
            cudaMemcpyAsync(mass, b->d_mass, (size_t)b->grids_cap * sizeof(double), cudaMemcpyDeviceToDevice,
                            b->stream);
        pool_free(b, b->d_grids);
        pool_free(b, b->d_mass);
        b->d_grids = grids;
        b->d_mass = mass;
        b->grids_cap = cap;
    }
    auto live = [](const Slot &s) { return s.used && !s.retiring && (s.target < 0 || s.step < s.target); };
    int nitems = 0;
    for (const Slot &s : b->slots)
        if (live(s)) nitems += s.tiles_x * s.tiles_y;
    if (nitems > b->items_cap) {
        pool_free(b, b->d_items);
        pool_free(b, b->d_partials);
        b->d_items = nullptr;
        b->d_partials = nullptr;
        b->items_cap = 0;
        const int cap = nitems * 2;
        if (pool_alloc(b, &b->d_items, (size_t)cap * sizeof(int4)) != cudaSuccess ||
            pool_alloc(b, &b->d_partials, (size_t)cap * sizeof(double)) != cudaSuccess) {
            pool_free(b, b->d_items);
            b->d_items = nullptr;
            return bfail(b, DUGKS_ENOMEM, "batch work list");
        }
        b->items_cap = cap;
    }
    const size_t gbytes = (size_t)std::max(n, 1) * sizeof(BatchGrid<T>);
    const size_t ibytes = (size_t)std::max(nitems, 1) * sizeof(int4);
    void *hg = nullptr, *hi = nullptr;
    size_t hgs = 0, his = 0;
    if (pinned_get(b, gbytes, &hg, &hgs) != DUGKS_OK) return bfail(b, DUGKS_ENOMEM, "descriptor staging");
    if (pinned_get(b, ibytes, &hi, &his) != DUGKS_OK) {
        pinned_put(b, hg, hgs);
        return bfail(b, DUGKS_ENOMEM, "work-list staging");
    }
    BatchGrid<T> *G = static_cast<BatchGrid<T> *>(hg);
    int4 *I = static_cast<int4 *>(hi);
    const bool half = Store<T, ST>::deviation;
    int k = 0;
    for (int i = 0; i < n; i++) {
        Slot &s = b->slots[i];
        BatchGrid<T> &d = G[i];
        if (!s.used || s.retiring) {
            std::memset(&d, 0, sizeof d);
            d.step = 0;
            d.target = 0;   // frozen
            continue;
        }
        if (s.desc.size() != sizeof(BatchGrid<T>)) {   // tensor maps, pointers and shape: once per grid
            BatchGrid<T> e;
            std::memset(&e, 0, sizeof e);
            for (int q = 0; q < 2; q++) {
                e.X[q] = s.X[q];
                if (!encode_plane_map(&e.tmX[q], s.X[q], b->ssize, half, s.pitch, s.ny, s.plane, 9, g.box_w,
                                      g.box_h)) {
                    pinned_put(b, hg, hgs);
                    pinned_put(b, hi, his);
                    return bfail(b, DUGKS_ECUDA, "tensor map encoding failed");
                }
            }
            for (int q = 0; q < b->nphi; q++) {
                e.phi[q] = static_cast<T *>(s.phi[q]);
                if (!encode_plane_map(&e.tmPhi[q], s.phi[q], sizeof(T), false, s.pitch, s.ny, s.plane, 1, g.box_wt,
                                      g.box_h)) {
                    pinned_put(b, hg, hgs);
                    pinned_put(b, hi, his);
                    return bfail(b, DUGKS_ECUDA, "tensor map encoding failed");
                }
            }
            if (b->nphi == 2) e.tmPhi[2] = e.tmPhi[0];
            e.plane = s.plane;
            e.nx = s.nx;
            e.ny = s.ny;
            e.pitch = s.pitch;
            e.tiles_x = s.tiles_x;
            e.vel_kind = s.vel_kind;
            for (int q = 0; q < 3; q++) e.vp[q] = s.vel[q];
            s.desc.assign(reinterpret_cast<unsigned char *>(&e), reinterpret_cast<unsigned char *>(&e) + sizeof e);
        }
        std::memcpy(&d, s.desc.data(), sizeof d);
        d.step = s.step;
        d.target = s.target < 0 ? (long long)1 << 62 : s.target;
        d.item0 = k;
        d.nitems = 0;
        if (live(s)) {
            d.nitems = s.tiles_x * s.tiles_y;
            for (int by = 0; by < s.tiles_y; by++)
                for (int bx = 0; bx < s.tiles_x; bx++) I[k++] = make_int4(i, bx, by, 0);
        }
    }
    b->nitems = nitems;
    cudaError_t e = cudaSuccess;
    if (n > 0) e = cudaMemcpyAsync(b->d_grids, hg, (size_t)n * sizeof(BatchGrid<T>), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess && nitems > 0)
        e = cudaMemcpyAsync(b->d_items, hi, (size_t)nitems * sizeof(int4), cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
        e = launch_batch_factors<T>(static_cast<BatchGrid<T> *>(b->d_grids), n, b->p.cfl, b->stream);
    uint64_t t = 0;
    const int fr = e == cudaSuccess ? fence(b, &t) : DUGKS_ECUDA;
    if (fr == DUGKS_OK) {
        pinned_later(b, hg, hgs, t);
        pinned_later(b, hi, his, t);
    } else {
        cudaStreamSynchronize(b->stream);
        pinned_put(b, hg, hgs);
        pinned_put(b, hi, his);
    }
    if (e != cudaSuccess) return bcuda(b, e, "batch descriptors upload");
    if (fr != DUGKS_OK) return fr;
    b->dirty = false;
    return DUGKS_OK;
}

int rebuild(dugks_batch *b) {
    switch (b->p.precision) {
    case DUGKS_FP64: return rebuild_t<double, double>(b);
    case DUGKS_FP32: return rebuild_t<float, float>(b);
    default: return rebuild_t<float, __half>(b);
    }
}

template <typename T, typename ST>
cudaError_t launch_one_step(dugks_batch *b) {
    const BatchUniform<T> &u = *reinterpret_cast<const BatchUniform<T> *>(b->uniform.data());
    const FaceCoefs<T> &cf = *reinterpret_cast<const FaceCoefs<T> *>(b->coefs.data());
    BatchGrid<T> *G = static_cast<BatchGrid<T> *>(b->d_grids);
    cudaError_t e = Launch<T, ST>::batch_step(u, cf, G, b->d_items, b->nitems, b->d_partials, b->p.order, b->p.flux,
                                              b->variant, b->ctas, b->stream);
    if (e != cudaSuccess) return e;
    return launch_batch_advance<T>(G, (int)b->slots.size(), b->d_partials, b->d_mass, b->d_status, u.dt, b->stream);
}

cudaError_t one_step(dugks_batch *b) {
    switch (b->p.precision) {
    case DUGKS_FP64: return launch_one_step<double, double>(b);
    case DUGKS_FP32: return launch_one_step<float, float>(b);
    default: return launch_one_step<float, __half>(b);
    }
}

template <typename T, typename ST>
StepParams<T> slot_view(const dugks_batch *b, const Slot &s) {
    StepParams<T> q;
    std::memset(&q, 0, sizeof q);
    q.nx = s.nx;
    q.ny = s.ny;
    q.pitch = s.pitch;
    q.plane = s.plane;
    q.status = b->d_status;
    q.theta_c = (T)(-4.0 / (b->p.W * (b->p.phiA - b->p.phiB)));
    q.phiA = (T)b->p.phiA;
    q.phiB = (T)b->p.phiB;
    q.vel_kind = s.vel_kind;
    q.vp0 = (T)s.vel[0];
    q.vp1 = (T)s.vel[1];
    q.vp2 = (T)s.vel[2];
    q.qscale = (T)256.0;
    q.qinv = (T)(1.0 / 256.0);
    q.X = s.X[s.step & 1];
    if (Store<T, ST>::phi_plane) q.phi_cur = static_cast<const T *>(s.phi[(3 - (int)(s.step % 3)) % 3]);
    q.tile_w = TILE_X;
    q.tile_h = TILE_Y;
    q.tiles_x = (s.nx + TILE_X - 1) / TILE_X;
    return q;
}

// The initial equilibrium of a new grid, queued on the stream: the ghost-bordered
// field goes through pinned staging into a pool buffer that is freed in stream
// order after the init kernel.
template <typename T, typename ST>
int init_slot(dugks_batch *b, Slot &s, const double *phi0) {
    const size_t bytes = s.plane * sizeof(T);
    void *d_phi0 = nullptr;
    if (pool_alloc(b, &d_phi0, bytes) != cudaSuccess) return DUGKS_ENOMEM;
    void *h = nullptr;
    size_t hs = 0;
    if (pinned_get(b, bytes, &h, &hs) != DUGKS_OK) {
        pool_free(b, d_phi0);
        return DUGKS_ENOMEM;
    }
    fill_ghosted_plane(static_cast<T *>(h), phi0, s.nx, s.ny, s.pitch);
    cudaError_t e = cudaMemcpyAsync(d_phi0, h, bytes, cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess) {
        StepParams<T> q = slot_view<T, ST>(b, s);
        q.t = (T)0;
        q.out1 = s.X[0];
        q.phi_out = static_cast<T *>(s.phi[0]);
        e = Launch<T, ST>::init(q, static_cast<const T *>(d_phi0), (T)(0.5 * b->p.cfl), b->p.order, b->stream);
    }
    pool_free(b, d_phi0);
    uint64_t t = 0;
    if (e == cudaSuccess && fence(b, &t) == DUGKS_OK) {
        pinned_later(b, h, hs, t);
    } else {
        cudaStreamSynchronize(b->stream);
        cudaGetLastError();
        pinned_put(b, h, hs);
    }
    return e == cudaSuccess ? DUGKS_OK : bcuda(b, e, "batch init");
}

// device memory back to the pool in stream order; a pending read-out's host
// buffer waits for its fence
void free_slot(dugks_batch *b, Slot &s) {
    for (void *q : {s.X[0], s.X[1], s.phi[0], s.phi[1], s.phi[2]}) pool_free(b, q);
    if (s.pinned) pinned_later(b, s.pinned, s.pinned_bytes, s.ticket);
    s = Slot();
}

int check_common(const dugks_params *p) {
    if (!p) return DUGKS_EINVAL;
    if (!(p->W > 0) || !(p->M > 0) || !(p->cfl > 0) || p->cfl > 1.0) return DUGKS_EINVAL;
    if ((p->order != 2 && p->order != 3) || (p->flux != 0 && p->flux != 1) || p->stages != 2) return DUGKS_EINVAL;
    if (p->precision < DUGKS_FP64 || p->precision > DUGKS_FP16F) return DUGKS_EINVAL;
    if (!(p->phiA != p->phiB)) return DUGKS_EINVAL;
    return DUGKS_OK;
}

}  // namespace

extern "C" {

int dugks_batch_create(const dugks_params *common, void *cuda_stream, dugks_batch **out) {
    if (!out) return DUGKS_EINVAL;
    *out = nullptr;
    int r = check_common(common);
    if (r != DUGKS_OK) return r;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
        cudaGetLastError();
        return DUGKS_ECUDA;
    }
    if (!encode_fn()) return DUGKS_ECUDA;
    dugks_batch *b = new dugks_batch();
    b->p = *common;
    cudaGetDevice(&b->dev);
    if (cuda_stream) {
        b->stream = static_cast<cudaStream_t>(cuda_stream);
    } else if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess) {
        b->own_stream = true;
    } else {
        delete b;
        return DUGKS_ECUDA;
    }
    b->tsize = fp64(b) ? 8 : 4;
    b->ssize = common->precision == DUGKS_FP64 ? 8 : common->precision == DUGKS_FP32 ? 4 : 2;
    b->nphi = common->precision == DUGKS_FP64 ? 2 : 3;   // FP32 and FP16F: phi is a plane of its own
    if (common->precision == DUGKS_FP32) b->variant = 5;
    if (const char *ev = std::getenv("DUGKS_FAST_VARIANT")) {
        const int v = std::atoi(ev);
        if (v >= 0 && v < FAST_VARIANTS) b->variant = v;
    }
    int pools = 0;
    cudaDeviceGetAttribute(&pools, cudaDevAttrMemoryPoolsSupported, b->dev);
    cudaMemPoolProps props;
    std::memset(&props, 0, sizeof props);
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = b->dev;
    if (!pools || cudaMemPoolCreate(&b->pool, &props) != cudaSuccess) {
        cudaGetLastError();
        b->pool = nullptr;
        dugks_batch_destroy(b);
        return DUGKS_ECUDA;
    }
    if (dev_malloc(&b->d_status, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        dugks_batch_destroy(b);
        return DUGKS_ENOMEM;
    }
    cudaMemset(b->d_status, 0, sizeof(int));
    b->ctas = resident_ctas(b);
    if (fp64(b)) fill_uniform<double>(b, batch_geom(b));
    else fill_uniform<float>(b, batch_geom(b));
    *out = b;
    return DUGKS_OK;
}

size_t dugks_batch_grid_bytes(const dugks_params *common, int32_t nx, int32_t ny) {
    if (!common || nx < 8 || ny < 8) return 0;
    const size_t plane = plane_of(nx, ny, nullptr);
    const size_t ts = common->precision == DUGKS_FP64 ? 8 : 4;
    const size_t ss = common->precision == DUGKS_FP64 ? 8 : common->precision == DUGKS_FP32 ? 4 : 2;
    const int nphi = common->precision == DUGKS_FP64 ? 2 : 3;
    return 2 * 9 * plane * ss + (size_t)nphi * plane * ts;
}

int dugks_batch_add(dugks_batch *b, int32_t nx, int32_t ny, const double *phi0_host, int vel_kind,
                    const double *vel_params, int64_t target_steps, int32_t *grid_id) {
    if (!b || !phi0_host || !grid_id || nx < 8 || ny < 8) return DUGKS_EINVAL;
    if (b->sticky != DUGKS_OK) return b->sticky;
    if (vel_kind != DUGKS_VEL_UNIFORM && vel_kind != DUGKS_VEL_ROTATION && vel_kind != DUGKS_VEL_VORTEX)
        return bfail(b, DUGKS_EINVAL, "batch grids take uniform, rotation or vortex velocity");
    if (!vel_params) return bfail(b, DUGKS_EINVAL, "velocity parameters missing");
    if (vel_kind == DUGKS_VEL_VORTEX && (!(vel_params[0] > 0) || !(vel_params[2] > 0)))
        return bfail(b, DUGKS_EINVAL, "vortex needs (L > 0, U, T > 0)");
    for (size_t i = 0; i < (size_t)nx * ny; i++)
        if (!std::isfinite(phi0_host[i])) return DUGKS_ENONFINITE;
    cudaSetDevice(b->dev);
    int r = advance(b);
    if (r != DUGKS_OK) return r;
    Slot s;
    s.used = true;
    s.nx = nx;
    s.ny = ny;
    s.plane = plane_of(nx, ny, &s.pitch);
    const FastGeom g = batch_geom(b);
    s.tiles_x = (nx + g.tile_w - 1) / g.tile_w;
    s.tiles_y = (ny + g.tile_h - 1) / g.tile_h;
    s.vel_kind = vel_kind;
    const int nv = vel_kind == DUGKS_VEL_UNIFORM ? 2 : 3;
    for (int k = 0; k < nv; k++) s.vel[k] = vel_params[k];
    s.target = target_steps;
    bool ok = true;
    for (int k = 0; k < 2 && ok; k++) ok = pool_alloc(b, &s.X[k], 9 * s.plane * b->ssize) == cudaSuccess;
    for (int k = 0; k < b->nphi && ok; k++) ok = pool_alloc(b, &s.phi[k], s.plane * b->tsize) == cudaSuccess;
    if (!ok) {
        free_slot(b, s);
        return DUGKS_ENOMEM;   // not sticky: the caller may retry later
    }
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 2 && e == cudaSuccess; k++) e = cudaMemsetAsync(s.X[k], 0, 9 * s.plane * b->ssize, b->stream);
    for (int k = 0; k < b->nphi && e == cudaSuccess; k++)
        e = cudaMemsetAsync(s.phi[k], 0, s.plane * b->tsize, b->stream);
    if (e != cudaSuccess) {
        free_slot(b, s);
        return bcuda(b, e, "batch grid clear");
    }
    switch (b->p.precision) {
    case DUGKS_FP64: r = init_slot<double, double>(b, s, phi0_host); break;
    case DUGKS_FP32: r = init_slot<float, float>(b, s, phi0_host); break;
    default: r = init_slot<float, __half>(b, s, phi0_host); break;
    }
    if (r != DUGKS_OK) {
        free_slot(b, s);
        return r;
    }
    int id = -1;
    for (size_t i = 0; i < b->slots.size(); i++)
        if (!b->slots[i].used) {
            id = (int)i;
            break;
        }
    if (id < 0) {
        id = (int)b->slots.size();
        b->slots.push_back(Slot());
    }
    b->slots[id] = s;
    b->dirty = true;
    *grid_id = id;
    return DUGKS_OK;
}

int dugks_batch_remove(dugks_batch *b, int32_t grid_id) {
    if (!b || grid_id < 0 || grid_id >= (int)b->slots.size() || !b->slots[grid_id].used) return DUGKS_EINVAL;
    cudaSetDevice(b->dev);
    free_slot(b, b->slots[grid_id]);
    b->dirty = true;
    return advance(b);
}

int dugks_batch_retire(dugks_batch *b, int32_t grid_id, uint64_t *ticket) {
    if (!b || !ticket || grid_id < 0 || grid_id >= (int)b->slots.size() || !b->slots[grid_id].used ||
        b->slots[grid_id].retiring)
        return DUGKS_EINVAL;
    if (b->sticky != DUGKS_OK) return b->sticky;
    cudaSetDevice(b->dev);
    Slot &s = b->slots[grid_id];
    const size_t bytes = (size_t)s.nx * s.ny * sizeof(double);
    void *h = nullptr;
    size_t hs = 0;
    if (pinned_get(b, bytes, &h, &hs) != DUGKS_OK) return DUGKS_ENOMEM;   // not sticky
    // phi widened to FP64 into the state set the last step read (no longer needed:
    // 9 planes of at least 2 bytes hold ny * nx doubles), then one copy to the host
    double *d = static_cast<double *>(s.X[1 - (int)(s.step & 1)]);
    cudaError_t e;
    switch (b->p.precision) {
    case DUGKS_FP64: e = Launch<double, double>::phi64(slot_view<double, double>(b, s), d, b->stream); break;
    case DUGKS_FP32: e = Launch<float, float>::phi64(slot_view<float, float>(b, s), d, b->stream); break;
    default: e = Launch<float, __half>::phi64(slot_view<float, __half>(b, s), d, b->stream); break;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, b->stream);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(b->stream);
        cudaGetLastError();
        pinned_put(b, h, hs);
        return bcuda(b, e, "retire read-out");
    }
    uint64_t t = 0;
    int r = fence(b, &t);
    if (r != DUGKS_OK) {
        cudaStreamSynchronize(b->stream);
        pinned_put(b, h, hs);
        return r;
    }
    s.retiring = true;
    s.target = s.step;   // frozen where it stands
    s.ticket = t;
    s.pinned = h;
    s.pinned_bytes = hs;
    b->dirty = true;
    *ticket = t;
    return DUGKS_OK;
}

int dugks_batch_collect(dugks_batch *b, int32_t grid_id, double *out_host, int wait) {
    if (!b || !out_host || grid_id < 0 || grid_id >= (int)b->slots.size() || !b->slots[grid_id].used ||
        !b->slots[grid_id].retiring)
        return DUGKS_EINVAL;
    cudaSetDevice(b->dev);
    Slot &s = b->slots[grid_id];
    int r = advance(b);
    if (r != DUGKS_OK) return r;
    if (b->reached < s.ticket) {
        if (!wait) return DUGKS_EAGAIN;
        r = wait_ticket(b, s.ticket);
        if (r != DUGKS_OK) return r;
    }
    if (b->sticky != DUGKS_OK) return b->sticky;
    std::memcpy(out_host, s.pinned, (size_t)s.nx * s.ny * sizeof(double));
    pinned_put(b, s.pinned, s.pinned_bytes);
    s.pinned = nullptr;
    free_slot(b, s);
    b->dirty = true;
    return DUGKS_OK;
}

int dugks_batch_fence(dugks_batch *b, uint64_t *ticket) {
    if (!b || !ticket) return DUGKS_EINVAL;
    if (b->sticky != DUGKS_OK) return b->sticky;
    cudaSetDevice(b->dev);
    return fence(b, ticket);
}

int dugks_batch_reached(dugks_batch *b, uint64_t ticket, int32_t *done) {
    if (!b || !done || ticket >= b->next_ticket) return DUGKS_EINVAL;
    cudaSetDevice(b->dev);
    const int r = advance(b);
    *done = b->reached >= ticket ? 1 : 0;
    return r;
}

int dugks_batch_set_ctas(dugks_batch *b, int32_t ctas) {
    if (!b) return DUGKS_EINVAL;
    cudaSetDevice(b->dev);
    b->ctas_req = ctas;
    b->ctas = ctas == 0 ? resident_ctas(b) : ctas < 0 ? INT_MAX : ctas;
    drop_graph(b);   // the next replay is captured with the new grid size
    return DUGKS_OK;
}

int dugks_batch_step(dugks_batch *b, int64_t nsteps) {
    if (!b || nsteps < 0) return DUGKS_EINVAL;
    if (b->sticky != DUGKS_OK) return b->sticky;
    cudaSetDevice(b->dev);
    int ar = advance(b);
    if (ar != DUGKS_OK) return ar;
    if (b->dirty) {
        int r = rebuild(b);
        if (r != DUGKS_OK) return r;
    }
    int64_t left = nsteps;
    cudaError_t e = cudaSuccess;
    while (left > 0 && e == cudaSuccess) {
        if (left >= GRAPH_STEPS) {
            if (!b->graph) {   // capture GRAPH_STEPS steps once; replayed while the work list is unchanged
                cudaGraph_t g = nullptr;
                e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
                for (int i = 0; i < GRAPH_STEPS && e == cudaSuccess; i++) e = one_step(b);
                cudaError_t e2 = cudaStreamEndCapture(b->stream, &g);
                if (e == cudaSuccess) e = e2;
                if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph, g, 0);
                if (g) cudaGraphDestroy(g);
                if (e != cudaSuccess) break;
            }
            e = cudaGraphLaunch(b->graph, b->stream);
            left -= GRAPH_STEPS;
            for (auto &s : b->slots)
                if (s.used) s.step = s.target < 0 ? s.step + GRAPH_STEPS : std::min(s.target, s.step + GRAPH_STEPS);
        } else {
            e = one_step(b);
            left -= 1;
            for (auto &s : b->slots)
                if (s.used && (s.target < 0 || s.step < s.target)) s.step += 1;
        }
    }
    if (e != cudaSuccess) return bcuda(b, e, "batch step");
    for (auto &s : b->slots)
        if (s.used && s.step > 0) s.mass_known = true;
    return DUGKS_OK;
}

int64_t dugks_batch_step_index(const dugks_batch *b, int32_t grid_id) {
    if (!b || grid_id < 0 || grid_id >= (int)b->slots.size() || !b->slots[grid_id].used) return -1;
    return b->slots[grid_id].step;
}

int64_t dugks_batch_active_cells(const dugks_batch *b) {
    if (!b) return 0;
    int64_t n = 0;
    for (auto &s : b->slots)
        if (s.used && (s.target < 0 || s.step < s.target)) n += (int64_t)s.nx * s.ny;
    return n;
}

int dugks_batch_read_phi(dugks_batch *b, int32_t grid_id, double *out_host) {
    if (!b || !out_host || grid_id < 0 || grid_id >= (int)b->slots.size() || !b->slots[grid_id].used)
        return DUGKS_EINVAL;
    if (b->sticky != DUGKS_OK) return b->sticky;
    cudaSetDevice(b->dev);
    const Slot &s = b->slots[grid_id];
    const size_t n = (size_t)s.nx * s.ny, bytes = n * sizeof(double);
    if (bytes > b->tmp_bytes) {
        cudaStreamSynchronize(b->stream);
        if (b->d_tmp) cudaFree(b->d_tmp);
        b->d_tmp = nullptr;
        b->tmp_bytes = 0;
        if (dev_malloc(&b->d_tmp, bytes) != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, DUGKS_ENOMEM, "read-out buffer");
        }
        b->tmp_bytes = bytes;
    }
    // phi widened to double on the device, then one copy into the caller's buffer
    cudaError_t e;
    double *d = static_cast<double *>(b->d_tmp);
    switch (b->p.precision) {
    case DUGKS_FP64: e = Launch<double, double>::phi64(slot_view<double, double>(b, s), d, b->stream); break;
    case DUGKS_FP32: e = Launch<float, float>::phi64(slot_view<float, float>(b, s), d, b->stream); break;
    default: e = Launch<float, __half>::phi64(slot_view<float, __half>(b, s), d, b->stream); break;
    }
    if (e != cudaSuccess) return bcuda(b, e, "phi kernel");
    e = cudaMemcpyAsync(out_host, d, bytes, cudaMemcpyDeviceToHost, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    return e == cudaSuccess ? b->sticky : bcuda(b, e, "read phi");
}

int dugks_batch_mass(dugks_batch *b, int32_t grid_id, double *out) {
    if (!b || !out || grid_id < 0 || grid_id >= (int)b->slots.size() || !b->slots[grid_id].used) return DUGKS_EINVAL;
    if (b->sticky != DUGKS_OK) return b->sticky;
    cudaSetDevice(b->dev);
    const Slot &s = b->slots[grid_id];
    cudaError_t e;
    if (s.mass_known && b->d_mass) {
        e = cudaMemcpyAsync(out, b->d_mass + grid_id, sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    } else {
        // before the first step: reduce the initial state with the generic tiling
        const int tiles = ((s.nx + TILE_X - 1) / TILE_X) * ((s.ny + TILE_Y - 1) / TILE_Y);
        const size_t need = (size_t)tiles * sizeof(double) + sizeof(double);
        if (need > b->tmp_bytes) {
            cudaStreamSynchronize(b->stream);
            if (b->d_tmp) cudaFree(b->d_tmp);
            b->d_tmp = nullptr;
            b->tmp_bytes = 0;
            if (dev_malloc(&b->d_tmp, need) != cudaSuccess) {
                cudaGetLastError();
                return bfail(b, DUGKS_ENOMEM, "mass buffer");
            }
            b->tmp_bytes = need;
        }
        double *part = static_cast<double *>(b->d_tmp), *res = part + tiles;
        switch (b->p.precision) {
        case DUGKS_FP64: { auto q = slot_view<double, double>(b, s); q.mass_partial = part; e = Launch<double, double>::mass_partial(q, b->stream); break; }
        case DUGKS_FP32: { auto q = slot_view<float, float>(b, s); q.mass_partial = part; e = Launch<float, float>::mass_partial(q, b->stream); break; }
        default: { auto q = slot_view<float, __half>(b, s); q.mass_partial = part; e = Launch<float, __half>::mass_partial(q, b->stream); break; }
        }
        if (e == cudaSuccess) e = launch_mass_final(part, tiles, res, b->d_status, b->stream);
        if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, sizeof(double), cudaMemcpyDeviceToHost, b->stream);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch mass");
    if (!std::isfinite(*out)) return bfail(b, DUGKS_ENONFINITE, "the field holds NaN or Inf");
    return DUGKS_OK;
}

int dugks_batch_set_variant(dugks_batch *b, int variant) {
    if (!b || variant < 0 || variant >= FAST_VARIANTS) return DUGKS_EINVAL;
    cudaSetDevice(b->dev);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch synchronize");
    b->variant = variant;
    b->ctas = b->ctas_req == 0 ? resident_ctas(b) : b->ctas_req < 0 ? INT_MAX : b->ctas_req;
    const FastGeom g = batch_geom(b);
    if (fp64(b)) fill_uniform<double>(b, g);
    else fill_uniform<float>(b, g);
    for (auto &s : b->slots)
        if (s.used) {
            s.tiles_x = (s.nx + g.tile_w - 1) / g.tile_w;
            s.tiles_y = (s.ny + g.tile_h - 1) / g.tile_h;
            s.desc.clear();   // tensor-map boxes follow the tile shape
        }
    b->dirty = true;
    return DUGKS_OK;
}

int dugks_batch_status(dugks_batch *b) {
    if (!b) return DUGKS_EINVAL;
    cudaSetDevice(b->dev);
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch synchronize");
    int flags = 0;
    e = cudaMemcpy(&flags, b->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return bcuda(b, e, "read status");
    if (flags & 2) return bfail(b, DUGKS_ETIMEOUT, "a device wait ran out");
    if (flags & 1) return bfail(b, DUGKS_ENONFINITE, "a grid holds NaN or Inf");
    return b->sticky;
}

const char *dugks_batch_last_error(const dugks_batch *b) { return b ? b->err.c_str() : "null batch"; }

void dugks_batch_destroy(dugks_batch *b) {
    if (!b) return;
    cudaSetDevice(b->dev);
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->graph) cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    for (auto &g : b->graphs_later) cudaGraphExecDestroy(g.second);
    if (b->pool) {
        for (auto &s : b->slots) free_slot(b, s);
        for (void *q : {b->d_grids, (void *)b->d_items, (void *)b->d_partials, (void *)b->d_mass}) pool_free(b, q);
        cudaStreamSynchronize(b->stream);
    }
    for (void *q : {(void *)b->d_status, b->d_tmp})
        if (q) cudaFree(q);
    for (auto &f : b->fences) cudaEventDestroy(f.second);
    for (cudaEvent_t ev : b->spare_events) cudaEventDestroy(ev);
    for (auto &q : b->pinned_later) cudaFreeHost(std::get<1>(q));
    for (auto &q : b->pinned_free) cudaFreeHost(q.second);
    if (b->pool) cudaMemPoolDestroy(b->pool);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"
