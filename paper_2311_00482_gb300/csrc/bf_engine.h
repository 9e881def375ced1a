// Host-side structures of the beamformer library (handles, plans, scratch,
// launch descriptions, serving engine).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <condition_variable>
#include <cstddef>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/bf.h"
#include "bf_internal.h"
#include "bf_tables.h"

namespace bfi {

int fail(int code, const char *fmt, ...);
int cuda_fail(cudaError_t e, const char *what);

// Owning device allocation (freed on destruction).
// Host-side fault injection for tests of the error paths: true when the
// environment variable BF_FAULT, a comma-separated list, names `kind`.
// Kinds: alloc (device allocations fail with BF_ENOMEM), submit (admission
// refuses every request with BF_EAGAIN), copy (a request's RF copy fails
// with BF_ECUDA).  Read on every use, so a test can switch it on and off.
bool fault_injected(const char *kind);

struct DevMem {
    void *p = nullptr;
    size_t bytes = 0;
    DevMem() = default;
    DevMem(const DevMem &) = delete;
    DevMem &operator=(const DevMem &) = delete;
    DevMem(DevMem &&o) noexcept : p(o.p), bytes(o.bytes)
    {
        o.p = nullptr;
        o.bytes = 0;
    }
    DevMem &operator=(DevMem &&o) noexcept
    {
        if (this != &o) {
            release();
            p = o.p;
            bytes = o.bytes;
            o.p = nullptr;
            o.bytes = 0;
        }
        return *this;
    }
    ~DevMem() { release(); }
    int ensure(size_t n);  // grow to at least n bytes (contents not kept)
    int reserve(size_t n); // as ensure, growing by half again at least (lists that vary in size)
    void release();
    int upload(const void *src, size_t n);  // synchronous host -> device
};

struct PlanKey {
    int ns, prec;
    std::vector<double> angles;
    int cfg = 0;  // index into kTileConfigs
    bool operator<(const PlanKey &o) const
    {
        if (ns != o.ns)
            return ns < o.ns;
        if (prec != o.prec)
            return prec < o.prec;
        if (cfg != o.cfg)
            return cfg < o.cfg;
        return angles < o.angles;
    }
};

// Device tables of one (handle, sample count, precision, angle set): the
// transmit tables, the counted-row intervals, the per-tile window starts and
// the tensor maps through which the beamformer stages its per-tile tables.
struct Plan {
    int ns = 0, na = 0, prec = 0;
    int wmax = 0, box = 0, group = 1, nsp = 0, rows = 8, tiles_x = 0, tiles_z = 0;
    DevMem colK, colF, rowK, rowF, valid, wtab, btab;
    DevMem maps;  // CUtensorMap[2]: valid rows, dx^2
};

struct EnvTablesDev {
    int nz = 0, fft_m = 0, bluestein = 0;
    DevMem tw, chirp, bhat;
};

// Device scratch of one in-flight frame: staged sample pairs, beamformed
// image, envelope, frame maxima and the tensor map over the pairs.
struct FrameScratch {
    DevMem pairs, y, env, maxbits, map;
    CUtensorMap map_host{};
    void *map_base = nullptr;
    int map_rows = 0, map_nsp = 0, map_box = 0, map_prec = -1;
    bool map_dirty = false;
    // as the lead of a multi-frame job: pairs holds the job's frames interleaved
    // ([row][pair][frame]) and map_nf describes that layout
    DevMem map_nf;
    CUtensorMap map_nf_host{};
    void *mapnf_base = nullptr;
    int mapnf_rows = 0, mapnf_nsp = 0, mapnf_box = 0, mapnf_prec = -1, mapnf_nf = 0;
    bool mapnf_dirty = false;
};

struct FramePrep {
    bf_handle *h = nullptr;
    Plan *plan = nullptr;
    std::shared_ptr<EnvTablesDev> et;   // envelope transform tables (nz)
    std::shared_ptr<EnvTablesDev> dt;   // demodulation transform tables (n_samples; IQ only)
    const int16_t *rf = nullptr;
    int ns = 0, na = 0, modes = 0, stage = 0, prec = 0;
    double pdas_p = 2.0;
    float *out = nullptr;
    void *pairs = nullptr;
    float *y = nullptr, *env = nullptr;
    unsigned *maxbits = nullptr;
    CUtensorMap *map_dev = nullptr;
    CUtensorMap map_host{};
    bool map_dirty = false;
    FrameScratch *scratch = nullptr;
    int nf_cap = 1;  // frames of a job this frame may lead (its pairs buffer holds that many)
};

struct HostLaunch {
    struct Group {  // one beamforming launch
        int prec, variant, rows, nf, first, count, prefix_first, tiles;
        size_t smem;
    };
    struct IGroup {  // one ingest launch
        int prec, first, count, prefix_first, rows;  // rows: the launch's CTAs
    };
    std::vector<BfJob> jobs;
    std::vector<int> tile_prefix;
    std::vector<Group> groups;
    size_t smem = 0;
    std::vector<IngestJob> ingest;
    std::vector<int> ingest_prefix;
    std::vector<IGroup> igroups;
    std::vector<EnvJob> env;
    std::vector<int> env_prefix;
    int env_blocks = 0;
    size_t env_smem = 0;
    // 512-row images: the warp-per-column-pair envelope kernel (column pairs)
    std::vector<EnvJob> envw;
    std::vector<int> envw_prefix;
    int envw_pairs = 0;
    std::vector<LogJob> log;
    std::vector<int> blk_prefix;
    int log_blocks = 0;
    std::vector<DemodJob> demod;   // IQ frames: records to analytic-signal pairs
    std::vector<int> demod_prefix;
    int demod_rows = 0, demod_max_ns = 0;
    bool demod_pairs = false;  // some demodulation job covers a frame pair
};

struct DeviceLaunch {
    DevMem jobs, tile_prefix, ingest, ingest_prefix, env, env_prefix, log, blk_prefix, err;
    DevMem envw, envw_prefix;
    DevMem demod, demod_prefix;
    int upload(const HostLaunch &hl, cudaStream_t st, bool async);
};

struct Request;

// The last bf_beamform call of a handle, kept so that the same call again
// (same plan, flags, buffers, order p and stream) skips the host-side
// preparation and, from its second repetition on, replays one CUDA graph.
struct CallCache {
    bool valid = false;
    const Plan *plan = nullptr;
    uint32_t flags = 0;
    const int16_t *rf = nullptr;
    float *out = nullptr;
    int ns = 0, na = 0;
    double pdas_p = 0;
    cudaStream_t stream = nullptr;
    int hits = 0;
    std::vector<FramePrep> frames;
    HostLaunch hl;
    cudaGraphExec_t exec = nullptr;
    void clear()
    {
        if (exec)
            cudaGraphExecDestroy(exec);
        exec = nullptr;
        valid = false;
        hits = 0;
        frames.clear();
        hl = HostLaunch{};
    }
};

}  // namespace bfi

struct bf_handle {
    int device = 0;
    bfi::GeomHost g;
    bfi::GeometryHost geo;
    cudaStream_t stream = nullptr, own_stream = nullptr;
    bfi::DevMem rowZ, dx2, apcnt;
    int kb_lo = 1, kb_hi = 0;
    double pdas_p = 2.0;  // order of the pDAS combiner
    std::mutex mu;  // plans, tickets, slot pool
    std::map<bfi::PlanKey, std::unique_ptr<bfi::Plan>> plans;
    std::map<bfi::PlanKey, int> tuned;  // tile configuration bf_autotune chose (key cfg = 0)
    bfi::FrameScratch scratch;     // bf_beamform
    bfi::DeviceLaunch launch;      // bf_beamform
    bfi::CallCache call;           // bf_beamform's last call
    bfi::DevMem fk_D, fk_spec, fk_img, fk_beta, fk_max, fk_log, fk_logp;  // bf_fkmig scratch
    bfi::DevMem fk_i0, fk_aw;     // bf_fkmig mapping tables, for fk_key
    std::vector<double> fk_key;   // (n_samples, Stolt?, angles...) of the tables
    bool err_cleared = false;
    std::map<uint64_t, std::shared_ptr<bfi::Request>> tickets;
};

struct bf_batch {
    int device = 0;
    std::vector<bfi::FrameScratch> scratch;
    std::vector<bfi::FramePrep> frames;
    bfi::HostLaunch hl;
    bfi::DeviceLaunch dl;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t marks[4] = {nullptr, nullptr, nullptr, nullptr};
    int launches = 0;  // kernels one replay launches
};

namespace bfi {

// Plan of a frame with these arguments (`flags`: its mode and precision bits).
// cfg < 0: the configuration bf_autotune chose for this workload, else the
// default; a two-row configuration serves DAS / DMAS of RF records and
// IQ-DAS / BB-DMAS only (an explicit one is refused for other frames, a tuned
// one replaced by the default).
int handle_plan(bf_handle *h, int ns, const double *angles, int na, uint32_t flags, Plan **out,
                int cfg = -1);
int check_frame_args(bf_handle *h, int ns, const double *angles, int na, uint32_t flags);
size_t frame_out_bytes(const bf_handle *h, uint32_t flags);
// Storage code of a frame's staged records (kPrecIQ for the IQ combiners).
int frame_prec(uint32_t flags);
// nf_cap: frames of one plan a later build_launch may put in one job with
// this frame (1: alone, as a single bf_beamform call); the frame's scratch
// is sized for the multi-frame jobs its plan and combiners allow up to that.
int prepare_frame(bf_handle *h, const int16_t *rf_dev, int ns, const double *angles, int na,
                  uint32_t flags, float *out_dev, FrameScratch &s, FramePrep &fp, int cfg = -1,
                  int nf_cap = 1);
// Frames (at most cap) of one plan that can share a beamforming job with a
// frame of these flags (1 unless the combiners are DAS / DMAS of RF records
// or IQ-DAS / BB-DMAS; IQ frames with records above 4096 samples alone).
int job_frames_cap(const Plan *p, uint32_t flags, int cap);
void build_launch(const std::vector<FramePrep> &frames, HostLaunch &hl);
int upload_maps(std::vector<FramePrep> &frames, cudaStream_t st, bool async);
// Stage marks of a captured graph on a side branch: mark k is recorded on the
// side stream after it joins the capture behind stage k (fork[k] recorded on
// the capture stream), so each mark node depends on the work it closes and no
// kernel depends on a mark: the kernels keep direct edges.  Mark 0 is a root
// beside the first launch.  join brings the side branch back into the
// capture's origin stream at the end.
struct MarkBranch {
    cudaStream_t side = nullptr;
    cudaEvent_t fork[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t join = nullptr;
};
// marks (optional, 4 events): recorded before the ingest, before and after the
// beamforming launches, and after the last launch; in line on st, or (branch,
// inside a capture of st) on the branch's side stream.
int enqueue(const std::vector<FramePrep> &frames, const HostLaunch &hl, DeviceLaunch &dl,
            cudaStream_t st, cudaEvent_t *marks = nullptr, const MarkBranch *branch = nullptr);
int read_device_error(DeviceLaunch &dl, cudaStream_t st);
bool is_device_pointer(const void *p);
void engine_forget(bf_handle *h);

}  // namespace bfi
