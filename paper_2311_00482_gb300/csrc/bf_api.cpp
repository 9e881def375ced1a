// C ABI of the beamformer: handles, resident tables, scratch, batches and the
// asynchronous submit / poll path.  See include/bf.h for the contract.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "../../include/bf.h"
#include "bf_engine.h"

namespace bfi {

// ------------------------------------------------------------------ errors --

static thread_local std::string g_err;

int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? BF_ENOMEM : BF_ECUDA, "%s: %s", what,
                cudaGetErrorString(e));
}

// ------------------------------------------------------------- device mem --

bool fault_injected(const char *kind)
{
    const char *e = std::getenv("BF_FAULT");
    if (!e || !*e)
        return false;
    const size_t n = std::strlen(kind);
    for (const char *p = e;;) {
        const char *q = std::strchr(p, ',');
        const size_t len = q ? (size_t)(q - p) : std::strlen(p);
        if (len == n && std::strncmp(p, kind, n) == 0)
            return true;
        if (!q)
            return false;
        p = q + 1;
    }
}

int DevMem::ensure(size_t n)
{
    if (n <= bytes && p)
        return BF_OK;
    release();
    if (n == 0)
        return BF_OK;
    if (fault_injected("alloc"))
        return fail(BF_ENOMEM, "injected allocation failure (BF_FAULT=alloc)");
    cudaError_t e = cudaMalloc(&p, n);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return cuda_fail(e, "cudaMalloc");
    }
    bytes = n;
    return BF_OK;
}

int DevMem::reserve(size_t n)
{
    if (n <= bytes && p)
        return BF_OK;
    return ensure(std::max<size_t>({n, bytes + bytes / 2, 4096}));
}

void DevMem::release()
{
    if (p)
        cudaFree(p);
    p = nullptr;
    bytes = 0;
}

int DevMem::upload(const void *src, size_t n)
{
    int rc = ensure(n);
    if (rc)
        return rc;
    if (n == 0)
        return BF_OK;
    cudaError_t e = cudaMemcpy(p, src, n, cudaMemcpyHostToDevice);
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "cudaMemcpy (tables)");
}

// ------------------------------------------------------------- tensor map --

static PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

// 2-D tensor map over a row-major table of `rows` rows of `cols` elements of
// `elem` bytes (4 or 8), read in boxes of box_cols x box_rows; out-of-range
// elements read as zero.
static int encode_map(CUtensorMap *map, void *base, int rows, int cols, int elem, int box_cols,
                      int box_rows)
{
    auto enc = tensor_map_encoder();
    if (!enc)
        return fail(BF_ECUDA, "cuTensorMapEncodeTiled is not available from the driver");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * (cuuint64_t)elem};
    cuuint32_t boxd[2] = {(cuuint32_t)box_cols, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = enc(map, elem == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_UINT32,
                     2, base, dims, strides, boxd, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return fail(BF_ECUDA, "cuTensorMapEncodeTiled failed (%d): %d x %d of %d bytes, box %d x %d",
                    (int)r, rows, cols, elem, box_cols, box_rows);
    return BF_OK;
}

static int encode_pairs_map(CUtensorMap *map, void *base, int rows, int nsp, int box, int prec)
{
    const int k = pair_elems(prec);  // IQ pairs: two 8-byte elements each
    return encode_map(map, base, rows, nsp * k, pair_bytes(prec) / k, box * k, 1);
}

// Pairs per frame of one tensor copy of an nf-frame job's interleaved window
// ([pair][frame], wmax pairs): the largest divisor of wmax whose copy spans at
// most kMaxBox tensor elements (IQ pairs: two each) and a multiple of 16 bytes
// (0: none).
static int interleaved_box(int wmax, int nf, int prec)
{
    const int pb = pair_bytes(prec);
    if ((wmax * nf * pb) % 16 != 0)
        return 0;
    for (int d = std::min(wmax, kMaxBox / (nf * pair_elems(prec))); d >= 1; --d)
        if (wmax % d == 0 && (d * nf * pb) % 16 == 0)
            return d;
    return 0;
}

// -------------------------------------------------------- envelope tables --

static std::mutex g_env_mu;
static std::map<std::pair<int, int>, std::shared_ptr<EnvTablesDev>> g_env_cache;  // (device, nz)

static int env_tables(int nz, std::shared_ptr<EnvTablesDev> &out)
{
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(g_env_mu);
    auto it = g_env_cache.find({dev, nz});
    if (it != g_env_cache.end()) {
        out = it->second;
        return BF_OK;
    }
    EnvHost eh;
    envelope_tables(nz, eh);
    auto t = std::make_shared<EnvTablesDev>();
    t->nz = nz;
    t->fft_m = eh.fft_m;
    t->bluestein = eh.bluestein;
    int rc = t->tw.upload(eh.tw.data(), eh.tw.size() * sizeof(float));
    if (!rc && eh.bluestein)
        rc = t->chirp.upload(eh.chirp.data(), eh.chirp.size() * sizeof(float));
    if (!rc && eh.bluestein)
        rc = t->bhat.upload(eh.bhat.data(), eh.bhat.size() * sizeof(float));
    if (rc)
        return rc;
    g_env_cache[{dev, nz}] = t;
    out = t;
    return BF_OK;
}

// ------------------------------------------------------------------ plans --

// Tile configuration of a workload: what bf_autotune measured fastest for it,
// else entry 0 (4 rows per thread, 32-row tiles, three CTAs per SM, measured
// faster than 8 rows on every grid tried); BF_TILE_ROWS=8 forces entry 3,
// BF_TILE_ROWS=2 entry 6 (16-row tiles of up to 22 channels per stage; DAS /
// DMAS of RF records, IQ-DAS / BB-DMAS; others keep entry 0).
static int choose_cfg(const bf_handle *h, const PlanKey &key)
{
    if (const char *e = std::getenv("BF_TILE_ROWS")) {
        if (std::atoi(e) == 8)
            return 3;
        if (std::atoi(e) == 4)
            return 0;
        if (std::atoi(e) == 2)
            return 6;
    }
    auto it = h->tuned.find(key);
    return it == h->tuned.end() ? 0 : it->second;
}

int handle_plan(bf_handle *h, int ns, const double *angles, int na, uint32_t flags, Plan **out,
                int cfg)
{
    const int prec = frame_prec(flags);
    const bool narrow_ok = (flags & BF_MODE_MASK & ~(BF_DAS | BF_DMAS)) == 0;
    PlanKey key{ns, prec, std::vector<double>(angles, angles + na), 0};
    std::lock_guard<std::mutex> lk(h->mu);
    key.cfg = (cfg >= 0 && cfg < kNumTileConfigs) ? cfg : choose_cfg(h, key);
    if (kTileConfigs[key.cfg].rows == 2 && !narrow_ok) {
        if (cfg >= 0)
            return fail(BF_EINVAL, "two-row tiles serve DAS / DMAS and IQ-DAS / BB-DMAS only");
        key.cfg = 0;
    }
    auto it = h->plans.find(key);
    if (it != h->plans.end()) {
        *out = it->second.get();
        return BF_OK;
    }
    PlanHost ph;
    const TileConfig tc = kTileConfigs[key.cfg];
    angle_tables(h->g, h->geo, ns, key.angles, prec, tc.rows, tc.stage_bytes, ph);
    if (beamform_smem_bytes(ph.wmax, ph.group, prec, 1, ph.rows) > (size_t)kMaxSmemPerCta)
        return fail(BF_EINVAL,
                    "pixel spacing too coarse for the sample rate: one tile needs %d samples per channel",
                    ph.wmax);
    auto p = std::make_unique<Plan>();
    p->ns = ns;
    p->na = na;
    p->prec = prec;
    p->wmax = ph.wmax;
    p->box = ph.box;
    p->group = ph.group;
    p->nsp = ph.nsp;
    p->rows = ph.rows;
    p->tiles_x = (h->g.nx + kTileCols - 1) / kTileCols;
    p->tiles_z = (h->g.nz + tile_rows(ph.rows) - 1) / tile_rows(ph.rows);
    const int nxp = pad_cols(h->g.nx), ne = h->g.ne;
    int rc = p->colK.upload(ph.colK.data(), ph.colK.size() * sizeof(int));
    if (!rc) rc = p->colF.upload(ph.colF.data(), ph.colF.size() * sizeof(float));
    if (!rc) rc = p->rowK.upload(ph.rowK.data(), ph.rowK.size() * sizeof(int));
    if (!rc) rc = p->rowF.upload(ph.rowF.data(), ph.rowF.size() * sizeof(float));
    if (!rc) rc = p->valid.upload(ph.valid.data(), ph.valid.size() * sizeof(int));
    if (!rc) rc = p->wtab.ensure((size_t)na * p->tiles_x * p->tiles_z * ne * sizeof(int));
    if (!rc) rc = p->btab.ensure((size_t)na * p->tiles_x * p->tiles_z * ne * sizeof(int));
    if (rc)
        return rc;
    CUtensorMap maps[2];
    rc = encode_map(&maps[0], p->valid.p, na * ne, nxp, 8, kTileCols, p->group);
    if (!rc)
        rc = encode_map(&maps[1], h->dx2.p, ne, nxp, 4, kTileCols, p->group);
    if (!rc)
        rc = p->maps.upload(maps, sizeof maps);
    if (rc)
        return rc;
    // window starts of every (angle, tile, channel), once per plan
    PlanJob pj{};
    pj.colK = (const int *)p->colK.p;
    pj.colF = (const float *)p->colF.p;
    pj.rowK = (const int *)p->rowK.p;
    pj.rowF = (const float *)p->rowF.p;
    pj.rowZ = (const float *)h->rowZ.p;
    pj.valid = (const int2 *)p->valid.p;
    pj.dx2 = (const float *)h->dx2.p;
    pj.wtab = (int *)p->wtab.p;
    pj.btab = (int *)p->btab.p;
    pj.nx = h->g.nx;
    pj.nxp = nxp;
    pj.nz = h->g.nz;
    pj.na = na;
    pj.ne = ne;
    pj.rows = p->rows;
    pj.tiles_x = p->tiles_x;
    pj.tiles_z = p->tiles_z;
    pj.wmax = p->wmax;
    pj.align = ph.align;
    DevMem errw;
    rc = errw.ensure(sizeof(int));
    if (rc)
        return rc;
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    int herr = 0;
    e = cudaMemsetAsync(errw.p, 0, sizeof(int), st);
    if (e == cudaSuccess)
        e = launch_plan(pj, (int *)errw.p, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&herr, errw.p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (e != cudaSuccess)
        return cuda_fail(e, "window planner");
    if (herr)
        return fail(BF_ECUDA, "window planner: a tile's delays span more than %d samples", p->wmax);
    *out = p.get();
    h->plans.emplace(std::move(key), std::move(p));
    return BF_OK;
}

// ------------------------------------------------------- frame preparation --

static constexpr double kPi = 3.14159265358979323846;

static int popcount4(int m) { return (m & 1) + ((m >> 1) & 1) + ((m >> 2) & 1) + ((m >> 3) & 1); }

// Images one frame produces: one per selected RF or IQ combiner.
static int frame_images(uint32_t flags)
{
    return popcount4(flags & BF_MODE_MASK) + ((flags & BF_IQDAS) ? 1 : 0) +
           ((flags & BF_BBDMAS) ? 1 : 0);
}

int frame_prec(uint32_t flags)
{
    return (flags & BF_IQ_MASK) ? (int)kPrecIQ : (int)((flags & BF_PREC_MASK) >> 4);
}

int check_frame_args(bf_handle *h, int ns, const double *angles, int na, uint32_t flags)
{
    if (!h)
        return fail(BF_EINVAL, "null handle");
    if (ns < 2 || ns > (1 << 24))
        return fail(BF_EINVAL, "n_samples must be in [2, 2^24], got %d", ns);
    if (na < 1 || na > 256)
        return fail(BF_EINVAL, "n_angles must be in [1, 256], got %d", na);
    if (!angles)
        return fail(BF_EINVAL, "null angles");
    for (int a = 0; a < na; ++a)
        if (!std::isfinite(angles[a]) || std::fabs(angles[a]) >= 1.5707963267948966)
            return fail(BF_EINVAL, "angle %d (%g rad) outside (-pi/2, pi/2)", a, angles[a]);
    const int modes = flags & BF_MODE_MASK, iq = flags & BF_IQ_MASK;
    if (!modes && !iq)
        return fail(BF_EINVAL,
                    "no combiner selected (BF_DAS / BF_DMAS / BF_CF / BF_PDAS / BF_IQDAS / BF_BBDMAS)");
    if (flags & ~(uint32_t)(BF_MODE_MASK | BF_IQ_MASK | BF_PREC_MASK | BF_OUT_MASK))
        return fail(BF_EINVAL, "unknown bits in mode_and_flags 0x%x", flags);
    const int prec = (flags & BF_PREC_MASK) >> 4;
    if (prec > kPrecBF16)
        return fail(BF_EINVAL, "unknown precision bits");
    if (iq) {
        if (modes)
            return fail(BF_EINVAL, "IQ combiners cannot be combined with RF combiners in one call");
        if (prec != kPrecF32)
            return fail(BF_EINVAL, "IQ combiners use FP32 storage");
        if (ns < 4 || ns > 8192 || (ns & (ns - 1)) != 0)
            return fail(BF_EINVAL, "IQ combiners need a power-of-two n_samples in [4, 8192] (got %d)",
                        ns);
    }
    const int stage = flags & BF_OUT_MASK;
    if (stage != BF_OUT_RF && stage != BF_OUT_ENV && stage != BF_OUT_LOGDB)
        return fail(BF_EINVAL, "unknown output stage bits");
    if (stage != BF_OUT_RF && h->g.nz > 4096)
        return fail(BF_EINVAL, "envelope detection supports nz <= 4096 (got %d)", h->g.nz);
    if ((long long)na * h->g.ne > (1LL << 30))
        return fail(BF_EINVAL, "too many channel records");
    return BF_OK;
}

size_t frame_out_bytes(const bf_handle *h, uint32_t flags)
{
    return (size_t)frame_images(flags) * (size_t)h->g.nx * (size_t)h->g.nz * sizeof(float);
}

static int plan_frames_per_job(const Plan *p, int modes, int prec, int cap);

int prepare_frame(bf_handle *h, const int16_t *rf_dev, int ns, const double *angles, int na,
                  uint32_t flags, float *out_dev, FrameScratch &s, FramePrep &fp, int cfg,
                  int nf_cap)
{
    int rc = check_frame_args(h, ns, angles, na, flags);
    if (rc)
        return rc;
    const int prec = frame_prec(flags);
    const bool iq = prec == kPrecIQ;
    Plan *plan = nullptr;
    rc = handle_plan(h, ns, angles, na, flags, &plan, cfg);
    if (rc)
        return rc;
    const int modes = flags & (BF_MODE_MASK | BF_IQ_MASK), nm = frame_images(flags);
    const int stage = flags & BF_OUT_MASK;
    const size_t img = (size_t)h->g.nx * h->g.nz;
    const int rows = na * h->g.ne;
    // room for the frames of a job this frame may lead (interleaved pairs)
    const int cap = plan_frames_per_job(plan, modes, prec, nf_cap);
    rc = s.pairs.ensure((size_t)cap * rows * plan->nsp * pair_bytes(prec));
    if (!rc && cap > 1)
        rc = s.map_nf.ensure(sizeof(CUtensorMap));
    if (!rc && stage != BF_OUT_RF && !iq)  // IQ images are magnitudes already
        rc = s.y.ensure(nm * img * sizeof(float));
    if (!rc && stage == BF_OUT_LOGDB)
        rc = s.env.ensure(nm * img * sizeof(float));
    if (!rc)
        rc = s.maxbits.ensure(4 * sizeof(unsigned));
    if (!rc)
        rc = s.map.ensure(sizeof(CUtensorMap));
    if (rc)
        return rc;
    fp = FramePrep{};
    fp.h = h;
    fp.plan = plan;
    fp.rf = rf_dev;
    fp.ns = ns;
    fp.na = na;
    fp.modes = modes;
    fp.pdas_p = h->pdas_p;
    fp.stage = stage;
    fp.prec = prec;
    fp.out = out_dev;
    fp.pairs = s.pairs.p;
    if (iq) {  // the beamformer writes magnitudes: straight out, or into the log stage's input
        fp.y = stage == BF_OUT_LOGDB ? (float *)s.env.p : out_dev;
        fp.env = stage == BF_OUT_LOGDB ? (float *)s.env.p : nullptr;
    } else {
        fp.y = stage == BF_OUT_RF ? out_dev : (float *)s.y.p;
        fp.env = stage == BF_OUT_ENV ? out_dev : (stage == BF_OUT_LOGDB ? (float *)s.env.p : nullptr);
    }
    fp.maxbits = (unsigned *)s.maxbits.p;
    fp.map_dev = (CUtensorMap *)s.map.p;
    fp.nf_cap = cap;
    if (s.map_base != s.pairs.p || s.map_rows != rows || s.map_nsp != plan->nsp ||
        s.map_box != plan->box || s.map_prec != prec) {
        rc = encode_pairs_map(&s.map_host, s.pairs.p, rows, plan->nsp, plan->box, prec);
        if (rc)
            return rc;
        s.map_base = s.pairs.p;
        s.map_rows = rows;
        s.map_nsp = plan->nsp;
        s.map_box = plan->box;
        s.map_prec = prec;
        s.map_dirty = true;
    }
    fp.map_host = s.map_host;
    fp.map_dirty = s.map_dirty;
    fp.scratch = &s;
    if (stage != BF_OUT_RF && !iq) {
        rc = env_tables(h->g.nz, fp.et);
        if (rc)
            return rc;
    }
    if (iq) {
        rc = env_tables(ns, fp.dt);  // twiddles of the length-ns transforms
        if (rc)
            return rc;
    }
    return BF_OK;
}

// Host-side launch description of a set of frames (job arrays + prefixes).
// Frames can share one beamforming job (and every delay) when they use the
// same plan with the same combiners: DAS and / or DMAS of RF records, or
// IQ-DAS and / or BB-DMAS (which share the carrier phase as well), up to two
// frames on 32-row tiles and four on 16-row tiles.
static int plan_frames_per_job(const Plan *p, int modes, int prec, int cap)
{
    const int m = modes & (BF_MODE_MASK | BF_IQ_MASK);
    if ((m & ~(BF_DAS | BF_DMAS | BF_IQ_MASK)) != 0)
        return 1;
    if (prec == kPrecIQ && demod_smem_bytes(p->ns, true) > (size_t)kMaxSmemPerCta)
        return 1;  // a frame pair's demodulation does not fit one CTA
    for (int nf = p->rows == 2 ? 4 : p->rows == 4 ? 2 : 1; nf > 1; nf /= 2)
        if (nf <= cap &&
            beamform_smem_bytes(p->wmax, p->group, prec, nf, p->rows) <= (size_t)kMaxSmemPerCta &&
            interleaved_box(p->wmax, nf, prec) > 0)
            return nf;
    return 1;
}

int job_frames_cap(const Plan *p, uint32_t flags, int cap)
{
    return plan_frames_per_job(p, (int)(flags & (BF_MODE_MASK | BF_IQ_MASK)), frame_prec(flags), cap);
}

static int max_frames_per_job(const FramePrep &a)
{
    return plan_frames_per_job(a.plan, a.modes, a.prec, a.nf_cap);
}

// The lead frame's tensor map of its job's interleaved pairs, encoded when the
// layout changed (uploaded by upload_maps).
static int lead_map(const FramePrep &f, int nf, int box)
{
    FrameScratch &S = *f.scratch;
    const int rows = f.na * f.h->g.ne, nsp = f.plan->nsp;
    if (!S.map_nf.p)
        return fail(BF_EINVAL, "frame scratch has no multi-frame map");
    if (S.mapnf_base == f.pairs && S.mapnf_rows == rows && S.mapnf_nsp == nsp &&
        S.mapnf_box == box && S.mapnf_prec == f.prec && S.mapnf_nf == nf)
        return BF_OK;
    const int k = pair_elems(f.prec);  // IQ pairs: two 8-byte elements each
    int rc = encode_map(&S.map_nf_host, f.pairs, rows, nsp * nf * k, pair_bytes(f.prec) / k,
                        box * nf * k, 1);
    if (rc)
        return rc;
    S.mapnf_base = f.pairs;
    S.mapnf_rows = rows;
    S.mapnf_nsp = nsp;
    S.mapnf_box = box;
    S.mapnf_prec = f.prec;
    S.mapnf_nf = nf;
    S.mapnf_dirty = true;
    return BF_OK;
}

static bool shareable(const FramePrep &a, const FramePrep &b)
{
    const int m = a.modes & (BF_MODE_MASK | BF_IQ_MASK);
    return a.plan == b.plan && a.h == b.h && m == (b.modes & (BF_MODE_MASK | BF_IQ_MASK)) &&
           a.prec == b.prec && a.na == b.na && a.ns == b.ns;
}

void build_launch(const std::vector<FramePrep> &frames, HostLaunch &hl)
{
    hl = HostLaunch{};
    std::map<int, std::vector<BfJob>> groups;
    std::map<int, size_t> group_smem;
    std::vector<char> taken(frames.size(), 0);
    // frames riding in another frame's job (the lead, the first of them, carries
    // the job's ingest)
    std::vector<char> member(frames.size(), 0);
    std::vector<std::vector<size_t>> partners(frames.size());
    for (size_t fi = 0; fi < frames.size(); ++fi) {
        if (taken[fi])
            continue;
        const FramePrep &f = frames[fi];
        taken[fi] = 1;
        // partner frames of the same plan, if any: all ride in one job (1, 2 or 4 frames)
        const FramePrep *more[kMaxFramesPerJob - 1] = {};
        const int cap = max_frames_per_job(f);
        std::vector<size_t> cand;
        for (size_t gi = fi + 1; gi < frames.size() && (int)cand.size() + 1 < cap; ++gi)
            if (!taken[gi] && shareable(f, frames[gi]))
                cand.push_back(gi);
        const int avail = (int)cand.size() + 1;
        int nf = avail >= 4 ? 4 : avail >= 2 ? 2 : 1;
        const int box_nf = nf > 1 ? interleaved_box(f.plan->wmax, nf, f.prec) : 0;
        if (nf > 1 && lead_map(f, nf, box_nf) != BF_OK)
            nf = 1;  // no interleaved map: every frame alone
        for (int q = 0; q < nf - 1; ++q) {
            more[q] = &frames[cand[q]];
            taken[cand[q]] = 1;
            member[cand[q]] = 1;
            partners[fi].push_back(cand[q]);
        }
        const bf_handle *h = f.h;
        const Plan *p = f.plan;
        BfJob j{};
        j.colK = (const int *)p->colK.p;
        j.colF = (const float *)p->colF.p;
        j.rowK = (const int *)p->rowK.p;
        j.rowF = (const float *)p->rowF.p;
        j.rowZ = (const float *)h->rowZ.p;
        j.wtab = (const int *)p->wtab.p;
        j.btab = (const int *)p->btab.p;
        j.apcnt = (const uint16_t *)h->apcnt.p;
        j.rf_map = f.map_dev;
        j.valid_map = (const CUtensorMap *)p->maps.p;
        j.dx2_map = (const CUtensorMap *)p->maps.p + 1;
        j.y = f.y;
        j.nx = h->g.nx;
        j.nz = h->g.nz;
        j.na = f.na;
        j.ne = h->g.ne;
        j.wmax = p->wmax;
        j.box = p->box;
        j.group = p->group;
        j.rows = p->rows;
        // the IQ kernel reads its two combiners from the DAS / DMAS slots of the mode word
        j.modes = f.prec == kPrecIQ ? (((f.modes & BF_IQDAS) ? BF_DAS : 0) |
                                       ((f.modes & BF_BBDMAS) ? BF_DMAS : 0))
                                    : f.modes;
        j.tiles_x = p->tiles_x;
        j.tiles_z = p->tiles_z;
        j.out_scale = (f.prec == kPrecF32 || f.prec == kPrecIQ) ? 1.0f : 32768.0f;
        j.pdas_p = (float)f.pdas_p;
        j.pdas_inv_p = (float)(1.0 / f.pdas_p);
        const double r = h->g.f0 / h->g.fs;  // carrier cycles per sample
        j.iq_c1 = (float)(2.0 * kPi * r);
        j.iq_c2 = (float)(kPi * r);
        j.maxbits = (f.prec == kPrecIQ && f.stage == BF_OUT_LOGDB) ? f.maxbits : nullptr;
        for (int q = 0; q < kMaxFramesPerJob - 1; ++q) {
            j.y_more[q] = more[q] ? more[q]->y : nullptr;
            j.maxbits_more[q] = (more[q] && f.prec == kPrecIQ && more[q]->stage == BF_OUT_LOGDB)
                                    ? more[q]->maxbits
                                    : nullptr;
        }
        if (nf > 1) {  // the frames' pairs interleaved in the lead's scratch
            j.rf_map = (const CUtensorMap *)f.scratch->map_nf.p;
            j.box = box_nf;
        }
        const int variant =
            ((nf * 16 + p->rows) * 4 + f.prec) * 16 + (j.modes & (BF_DMAS | BF_CF | BF_PDAS));
        groups[variant].push_back(j);
        const size_t sm = beamform_smem_bytes(p->wmax, p->group, f.prec, nf, p->rows);
        group_smem[variant] = std::max(group_smem[variant], sm);
        hl.smem = std::max(hl.smem, sm);
    }
    for (auto &kv : groups) {
        HostLaunch::Group g;
        g.nf = kv.first / (16 * 4 * 16);
        g.rows = (kv.first / 64) % 16;
        g.prec = (kv.first / 16) % 4;
        g.variant = kv.first % 16;
        g.smem = group_smem[kv.first];
        g.first = (int)hl.jobs.size();
        g.count = (int)kv.second.size();
        g.prefix_first = (int)hl.tile_prefix.size();
        int acc = 0;
        for (const BfJob &j : kv.second) {
            hl.tile_prefix.push_back(acc);
            acc += j.tiles_x * j.tiles_z;
            hl.jobs.push_back(j);
        }
        g.tiles = acc;
        hl.groups.push_back(g);
    }
    std::map<int, std::vector<IngestJob>> ig;
    // IQ frames: one demodulation job per frame, or per frame pair of a
    // multi-frame job (into the lead's interleaved array)
    for (size_t fi = 0; fi < frames.size(); ++fi) {
        const FramePrep &f = frames[fi];
        if (f.prec != kPrecIQ || member[fi])
            continue;
        std::vector<size_t> job{fi};
        job.insert(job.end(), partners[fi].begin(), partners[fi].end());
        const int nf = (int)job.size();
        const double r = f.h->g.f0 / f.h->g.fs;
        for (int q = 0; q < (nf == 1 ? 1 : nf / 2); ++q) {
            const FramePrep &a = frames[job[nf == 1 ? 0 : 2 * q]];
            DemodJob d{};
            d.rf = a.rf;
            d.pairs = (float4 *)f.pairs;
            d.nf = nf;
            d.fi = nf == 1 ? 0 : 2 * q;
            d.rows = f.na * f.h->g.ne;
            d.ns = f.ns;
            d.nsp = f.plan->nsp;
            d.lgn = 0;
            while ((1 << d.lgn) < f.ns)
                ++d.lgn;
            d.rot = make_float2((float)std::cos(2.0 * kPi * r), (float)-std::sin(2.0 * kPi * r));
            d.tw = (const float2 *)f.dt->tw.p;
            d.maxbits = a.stage != BF_OUT_RF ? a.maxbits : nullptr;
            if (nf > 1) {
                const FramePrep &b = frames[job[2 * q + 1]];
                d.rf2 = b.rf;
                d.maxbits2 = b.stage != BF_OUT_RF ? b.maxbits : nullptr;
                hl.demod_pairs = true;
            }
            hl.demod_prefix.push_back(hl.demod_rows);
            hl.demod_rows += d.rows;
            hl.demod_max_ns = std::max(hl.demod_max_ns, f.ns);
            hl.demod.push_back(d);
        }
    }
    for (size_t fi = 0; fi < frames.size(); ++fi) {
        const FramePrep &f = frames[fi];
        if (f.prec == kPrecIQ || member[fi])
            continue;  // IQ frames demodulate; members of a job come with its lead
        IngestJob ij{};
        ij.rf = f.rf;
        ij.pairs = f.pairs;
        ij.rows = f.na * f.h->g.ne;
        ij.ns = f.ns;
        ij.nsp = f.plan->nsp;
        ij.maxbits = f.stage != BF_OUT_RF ? f.maxbits : nullptr;
        ij.nf = 1 + (int)partners[fi].size();
        if (ij.nf > 1) {  // the whole job, interleaved into the lead's pairs
            for (size_t q = 0; q < partners[fi].size(); ++q) {
                const FramePrep &g = frames[partners[fi][q]];
                ij.rf_more[q] = g.rf;
                ij.maxbits_more[q] = g.stage != BF_OUT_RF ? g.maxbits : nullptr;
            }
        }
        // threads per record row: one per 8 pairs and frame (per frame pair for
        // FP32 multi-frame jobs)
        const int units = (f.prec == kPrecF32 && ij.nf > 1) ? ij.nf / 2 : ij.nf;
        ij.chunks = (units * ((ij.nsp + 7) / 8) + 255) / 256;
        ig[f.prec].push_back(ij);
    }
    for (auto &kv : ig) {
        HostLaunch::IGroup g;
        g.prec = kv.first;
        g.first = (int)hl.ingest.size();
        g.count = (int)kv.second.size();
        g.prefix_first = (int)hl.ingest_prefix.size();
        int acc = 0;
        for (const IngestJob &j : kv.second) {
            hl.ingest_prefix.push_back(acc);  // first CTA of the job
            acc += j.rows * j.chunks;
            hl.ingest.push_back(j);
        }
        g.rows = acc;
        hl.igroups.push_back(g);
    }
    int cols = 0;
    long long blks = 0;
    for (const FramePrep &f : frames) {
        if (f.stage == BF_OUT_RF)
            continue;
        const bf_handle *h = f.h;
        const size_t img = (size_t)h->g.nx * h->g.nz;
        if (f.prec == kPrecIQ) {  // magnitude images: only the log stage follows
            if (f.stage != BF_OUT_LOGDB)
                continue;
            const int nimg = ((f.modes & BF_IQDAS) ? 1 : 0) + ((f.modes & BF_BBDMAS) ? 1 : 0);
            for (int slot = 0; slot < nimg; ++slot) {
                LogJob l{};
                l.env = f.env + slot * img;
                l.out = f.out + slot * img;
                l.maxbits = f.maxbits + slot;
                l.n = (int)img;
                l.vec4 = (img % 4 == 0 && ((uintptr_t)l.env & 15) == 0 && ((uintptr_t)l.out & 15) == 0)
                             ? 1
                             : 0;
                hl.blk_prefix.push_back((int)blks);
                blks += log_blocks((long long)img);
                hl.log.push_back(l);
            }
            continue;
        }
        int slot = 0;
        for (int bit = 1; bit <= BF_PDAS; bit <<= 1) {
            if (!(f.modes & bit))
                continue;
            EnvJob e{};
            e.y = f.y + slot * img;
            e.env = f.env + slot * img;
            e.maxbits = f.maxbits + slot;
            e.nx = h->g.nx;
            e.nz = h->g.nz;
            e.fft_m = f.et->fft_m;
            e.bluestein = f.et->bluestein;
            e.band = bit == BF_DMAS ? 1 : 0;
            e.kb_lo = h->kb_lo;
            e.kb_hi = h->kb_hi;
            e.tw = (const float2 *)f.et->tw.p;
            e.chirp = (const float2 *)f.et->chirp.p;
            e.bhat = (const float2 *)f.et->bhat.p;
            e.cols_per_block = e.bluestein ? 1 : envelope_cols_per_block(e.fft_m);
            e.vec4 = (!e.bluestein && e.nz % 4 == 0 && ((uintptr_t)e.y & 15) == 0 &&
                      ((uintptr_t)e.env & 15) == 0)
                         ? 1
                         : 0;
            if (envelope_warp_ok(e.nz, e.fft_m, e.bluestein)) {
                hl.envw_prefix.push_back(hl.envw_pairs);
                hl.envw_pairs += (h->g.nx + 1) / 2;
                hl.envw.push_back(e);
            } else {
                hl.env_prefix.push_back(cols);
                cols += (h->g.nx + e.cols_per_block - 1) / e.cols_per_block;
                hl.env.push_back(e);
                hl.env_smem = std::max(hl.env_smem, envelope_smem_bytes(e.fft_m, e.bluestein));
            }
            if (f.stage == BF_OUT_LOGDB) {
                LogJob l{};
                l.env = e.env;
                l.out = f.out + slot * img;
                l.maxbits = e.maxbits;
                l.n = (int)img;
                l.vec4 = (img % 4 == 0 && ((uintptr_t)l.env & 15) == 0 && ((uintptr_t)l.out & 15) == 0)
                             ? 1
                             : 0;
                hl.blk_prefix.push_back((int)blks);
                blks += log_blocks((long long)img);
                hl.log.push_back(l);
            }
            ++slot;
        }
    }
    hl.env_blocks = cols;
    hl.log_blocks = (int)blks;
}

int DeviceLaunch::upload(const HostLaunch &hl, cudaStream_t st, bool async)
{
    auto put = [&](DevMem &d, const void *src, size_t n) -> int {
        if (n == 0)
            return BF_OK;
        int rc = d.reserve(n);
        if (rc)
            return rc;
        cudaError_t e = async ? cudaMemcpyAsync(d.p, src, n, cudaMemcpyHostToDevice, st)
                              : cudaMemcpy(d.p, src, n, cudaMemcpyHostToDevice);
        return e == cudaSuccess ? BF_OK : cuda_fail(e, "cudaMemcpy (job list)");
    };
    int rc = put(jobs, hl.jobs.data(), hl.jobs.size() * sizeof(BfJob));
    if (!rc) rc = put(tile_prefix, hl.tile_prefix.data(), hl.tile_prefix.size() * sizeof(int));
    if (!rc) rc = put(ingest, hl.ingest.data(), hl.ingest.size() * sizeof(IngestJob));
    if (!rc) rc = put(ingest_prefix, hl.ingest_prefix.data(), hl.ingest_prefix.size() * sizeof(int));
    if (!rc) rc = put(env, hl.env.data(), hl.env.size() * sizeof(EnvJob));
    if (!rc) rc = put(env_prefix, hl.env_prefix.data(), hl.env_prefix.size() * sizeof(int));
    if (!rc) rc = put(envw, hl.envw.data(), hl.envw.size() * sizeof(EnvJob));
    if (!rc) rc = put(envw_prefix, hl.envw_prefix.data(), hl.envw_prefix.size() * sizeof(int));
    if (!rc) rc = put(log, hl.log.data(), hl.log.size() * sizeof(LogJob));
    if (!rc) rc = put(blk_prefix, hl.blk_prefix.data(), hl.blk_prefix.size() * sizeof(int));
    if (!rc) rc = put(demod, hl.demod.data(), hl.demod.size() * sizeof(DemodJob));
    if (!rc) rc = put(demod_prefix, hl.demod_prefix.data(), hl.demod_prefix.size() * sizeof(int));
    if (!rc) rc = err.ensure(sizeof(int));
    return rc;
}

// Tensor maps of frames whose scratch changed go to device memory (before any
// kernel reads them).
int upload_maps(std::vector<FramePrep> &frames, cudaStream_t st, bool async)
{
    auto copy = [&](void *dst, const CUtensorMap *src) -> int {
        cudaError_t e = async ? cudaMemcpyAsync(dst, src, sizeof(CUtensorMap),
                                                cudaMemcpyHostToDevice, st)
                              : cudaMemcpy(dst, src, sizeof(CUtensorMap), cudaMemcpyHostToDevice);
        return e == cudaSuccess ? BF_OK : cuda_fail(e, "cudaMemcpy (tensor map)");
    };
    for (FramePrep &f : frames) {
        FrameScratch &S = *f.scratch;
        if (f.map_dirty) {
            int rc = copy(f.map_dev, &S.map_host);
            if (rc)
                return rc;
            S.map_dirty = false;
            f.map_dirty = false;
        }
        if (S.mapnf_dirty) {  // the frame leads a multi-frame job
            int rc = copy(S.map_nf.p, &S.map_nf_host);
            if (rc)
                return rc;
            S.mapnf_dirty = false;
        }
    }
    return BF_OK;
}

// The device work of a set of frames, in stream order: ingest, reset of the
// frame maxima, beamforming (one launch per precision / combiner variant),
// envelope, log compression.
int enqueue(const std::vector<FramePrep> &frames, const HostLaunch &hl, DeviceLaunch &dl,
            cudaStream_t st, cudaEvent_t *marks, const MarkBranch *branch)
{
    cudaError_t e;
    // Inside a stream capture the marks must be external event records (they
    // become graph nodes that record at replay time); outside, plain records.
    // An event record between two kernels of a graph costs about 2 us and
    // keeps the next kernel from being launched ahead, so in a capture with a
    // branch the marks hang off a side stream instead.
    unsigned mark_flags = cudaEventRecordDefault;
    if (marks) {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(st, &cs);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaStreamIsCapturing");
        if (cs == cudaStreamCaptureStatusActive)
            mark_flags = cudaEventRecordExternal;
        else
            branch = nullptr;
    }
    auto mark = [&](int k) -> cudaError_t {
        if (!marks)
            return cudaSuccess;
        if (!branch)
            return cudaEventRecordWithFlags(marks[k], st, mark_flags);
        cudaError_t r = cudaEventRecord(branch->fork[k], st);
        if (r == cudaSuccess)
            r = cudaStreamWaitEvent(branch->side, branch->fork[k], 0);
        if (r == cudaSuccess)
            r = cudaEventRecordWithFlags(marks[k], branch->side, mark_flags);
        return r;
    };
    e = mark(0);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord (mark)");
    for (const HostLaunch::IGroup &g : hl.igroups) {
        e = launch_ingest((const IngestJob *)dl.ingest.p + g.first,
                          (const int *)dl.ingest_prefix.p + g.prefix_first, g.count, g.rows, g.prec,
                          st);
        if (e != cudaSuccess)
            return cuda_fail(e, "ingest launch");
    }
    if (!hl.demod.empty()) {
        e = launch_demod((const DemodJob *)dl.demod.p, (const int *)dl.demod_prefix.p,
                         (int)hl.demod.size(), hl.demod_rows, hl.demod_max_ns, hl.demod_pairs, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "demodulation launch");
    }
    // (the ingest / demodulation launches above zeroed each frame's image maxima)
    e = mark(1);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord (mark)");
    for (const HostLaunch::Group &g : hl.groups) {
        e = launch_beamform((const BfJob *)dl.jobs.p + g.first,
                            (const int *)dl.tile_prefix.p + g.prefix_first, g.count, g.tiles, g.smem,
                            g.prec, g.variant, g.rows, g.nf, (int *)dl.err.p, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "beamform launch");
    }
    e = mark(2);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord (mark)");
    if (!hl.env.empty()) {
        e = launch_envelope((const EnvJob *)dl.env.p, (const int *)dl.env_prefix.p, (int)hl.env.size(),
                            hl.env_blocks, hl.env_smem, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "envelope launch");
    }
    if (!hl.envw.empty()) {
        e = launch_envelope_warp((const EnvJob *)dl.envw.p, (const int *)dl.envw_prefix.p,
                                 (int)hl.envw.size(), hl.envw_pairs, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "envelope launch");
    }
    if (!hl.log.empty()) {
        e = launch_log((const LogJob *)dl.log.p, (const int *)dl.blk_prefix.p, (int)hl.log.size(),
                       hl.log_blocks, 70.0f, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "log launch");
    }
    e = mark(3);
    if (e == cudaSuccess && marks && branch) {  // the side branch back into st
        e = cudaEventRecord(branch->join, branch->side);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(st, branch->join, 0);
    }
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaEventRecord (mark)");
    return BF_OK;
}

int read_device_error(DeviceLaunch &dl, cudaStream_t st)
{
    int v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, dl.err.p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_fail(e, "reading the device status word");
    if (v) {
        cudaMemsetAsync(dl.err.p, 0, sizeof(int), st);
        if (v & kErrTimeout)
            return fail(BF_ETIMEDOUT, "a bounded device wait gave up (status 0x%x)", v);
        return fail(BF_ECUDA, "device-side check failed (status 0x%x)", v);
    }
    return BF_OK;
}

bool is_device_pointer(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace bfi

using namespace bfi;

// ===================================================================== ABI ==

extern "C" {

BF_API const char *bf_last_error(void) { return g_err.c_str(); }

BF_API int bf_version(void) { return 100; }

BF_API int bf_create(const bf_geometry *geom, const bf_grid *grid, double fs_hz, double f0_hz,
                     double c_mps, bf_handle **out)
{
    if (!geom || !grid || !out)
        return fail(BF_EINVAL, "null argument");
    *out = nullptr;
    const int ne = geom->n_elements;
    if (ne < 1 || ne > 4096)
        return fail(BF_EINVAL, "n_elements must be in [1, 4096], got %d", ne);
    if (!(geom->f_number > 0.0) || !std::isfinite(geom->f_number))
        return fail(BF_EINVAL, "f_number must be > 0");
    if (!geom->x_elem_m && !(geom->pitch_m > 0.0 && std::isfinite(geom->pitch_m)))
        return fail(BF_EINVAL, "pitch_m must be > 0 when x_elem_m is NULL");
    if (grid->nx < 1 || grid->nz < 1 || grid->nx > 32767 || grid->nz > 32767)
        return fail(BF_EINVAL, "grid dimensions must be in [1, 32767]");
    const double v[] = {grid->x0_m, grid->x1_m, grid->z0_m, grid->z1_m, fs_hz, f0_hz, c_mps};
    for (double d : v)
        if (!std::isfinite(d))
            return fail(BF_EINVAL, "non-finite grid or acquisition parameter");
    if (grid->x1_m < grid->x0_m || grid->z1_m < grid->z0_m || grid->z0_m < 0.0)
        return fail(BF_EINVAL, "grid must satisfy x1 >= x0 and z1 >= z0 >= 0");
    if (!(fs_hz > 0.0) || !(c_mps > 0.0) || !(f0_hz > 0.0))
        return fail(BF_EINVAL, "fs, f0 and c must be > 0");
    auto h = std::make_unique<bf_handle>();
    GeomHost &g = h->g;
    g.ne = ne;
    g.xe.resize(ne);
    for (int i = 0; i < ne; ++i)
        g.xe[i] = geom->x_elem_m ? geom->x_elem_m[i]
                                 : ((double)i - 0.5 * (double)(ne - 1)) * geom->pitch_m;
    for (int i = 0; i < ne; ++i) {
        if (!std::isfinite(g.xe[i]))
            return fail(BF_EINVAL, "non-finite element position");
        if (i && !(g.xe[i] > g.xe[i - 1]))
            return fail(BF_EINVAL, "element positions must be strictly increasing");
    }
    g.fnum = geom->f_number;
    g.nx = grid->nx;
    g.nz = grid->nz;
    g.x0 = grid->x0_m;
    g.x1 = grid->x1_m;
    g.z0 = grid->z0_m;
    g.z1 = grid->z1_m;
    g.fs = fs_hz;
    g.f0 = f0_hz;
    g.c = c_mps;
    cudaError_t e = cudaGetDevice(&h->device);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaGetDevice");
    e = cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    h->stream = h->own_stream;
    geometry_tables(g, h->geo);
    int rc = h->rowZ.upload(h->geo.rowZ.data(), h->geo.rowZ.size() * sizeof(float));
    if (!rc) rc = h->dx2.upload(h->geo.dx2.data(), h->geo.dx2.size() * sizeof(float));
    if (!rc) rc = h->apcnt.upload(h->geo.apcnt.data(), h->geo.apcnt.size() * sizeof(uint16_t));
    if (rc)
        return rc;
    bandpass_bins(g.nz, g.z0, g.z1, g.c, g.f0, h->kb_lo, h->kb_hi);
    *out = h.release();
    return BF_OK;
}

BF_API int bf_destroy(bf_handle *h)
{
    if (!h)
        return fail(BF_EINVAL, "null handle");
    {
        std::lock_guard<std::mutex> lk(h->mu);
        if (!h->tickets.empty())
            return fail(BF_EINVAL, "handle has %zu pending tickets", h->tickets.size());
    }
    cudaSetDevice(h->device);
    cudaStreamSynchronize(h->stream);
    h->call.clear();
    engine_forget(h);
    if (h->own_stream)
        cudaStreamDestroy(h->own_stream);
    delete h;
    return BF_OK;
}

BF_API int bf_set_stream(bf_handle *h, void *stream)
{
    if (!h)
        return fail(BF_EINVAL, "null handle");
    h->stream = stream ? (cudaStream_t)stream : h->own_stream;
    return BF_OK;
}

BF_API int bf_set_pdas_order(bf_handle *h, double p)
{
    if (!h)
        return fail(BF_EINVAL, "null handle");
    if (!(p >= 1.0 && p <= 16.0))
        return fail(BF_EINVAL, "pDAS order must be in [1, 16], got %g", p);
    h->pdas_p = p;
    return BF_OK;
}

BF_API size_t bf_output_bytes(const bf_handle *h, uint32_t flags)
{
    return h ? frame_out_bytes(h, flags) : 0;
}

BF_API int bf_beamform(bf_handle *h, const int16_t *rf_dev, int32_t n_samples,
                       const double *angles_rad, int32_t n_angles, uint32_t flags, float *out_dev)
{
    if (!h)
        return fail(BF_EINVAL, "null handle");
    if (!rf_dev || !out_dev)
        return fail(BF_EINVAL, "null data pointer");
    cudaSetDevice(h->device);
    CallCache &cc = h->call;
    if (cc.valid) {  // the same call as last time: no preparation, no uploads
        int rc = check_frame_args(h, n_samples, angles_rad, n_angles, flags);
        if (rc)
            return rc;
        Plan *plan = nullptr;
        rc = handle_plan(h, n_samples, angles_rad, n_angles, flags, &plan);
        if (rc)
            return rc;
        if (plan == cc.plan && flags == cc.flags && rf_dev == cc.rf && out_dev == cc.out &&
            n_samples == cc.ns && n_angles == cc.na && h->pdas_p == cc.pdas_p &&
            h->stream == cc.stream) {
            if (!cc.exec && ++cc.hits >= 1) {  // a repeat: capture the launches once
                cudaStream_t cap;
                cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
                if (e == cudaSuccess) {
                    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
                    if (e == cudaSuccess) {
                        rc = enqueue(cc.frames, cc.hl, h->launch, cap);
                        cudaGraph_t g = nullptr;
                        e = cudaStreamEndCapture(cap, &g);
                        if (!rc && e == cudaSuccess)
                            e = cudaGraphInstantiate(&cc.exec, g, 0);
                        if (g)
                            cudaGraphDestroy(g);
                        if (e != cudaSuccess || rc) {
                            cudaGetLastError();
                            cc.exec = nullptr;  // stay on the plain replay
                        }
                        rc = BF_OK;
                    }
                    cudaStreamDestroy(cap);
                }
                cudaGetLastError();
            }
            if (cc.exec) {
                cudaError_t e = cudaGraphLaunch(cc.exec, h->stream);
                return e == cudaSuccess ? BF_OK : cuda_fail(e, "cudaGraphLaunch");
            }
            return enqueue(cc.frames, cc.hl, h->launch, h->stream);
        }
    }
    cc.clear();
    if (!is_device_pointer(rf_dev) || !is_device_pointer(out_dev))
        return fail(BF_EINVAL, "bf_beamform needs device pointers (use bf_submit for host data)");
    std::vector<FramePrep> frames(1);
    int rc = prepare_frame(h, rf_dev, n_samples, angles_rad, n_angles, flags, out_dev, h->scratch,
                           frames[0]);
    if (rc)
        return rc;
    HostLaunch hl;
    build_launch(frames, hl);
    rc = upload_maps(frames, h->stream, true);
    if (!rc)
        rc = h->launch.upload(hl, h->stream, true);
    if (!rc && !h->err_cleared) {
        cudaMemsetAsync(h->launch.err.p, 0, sizeof(int), h->stream);
        h->err_cleared = true;
    }
    if (!rc)
        rc = enqueue(frames, hl, h->launch, h->stream);
    if (!rc) {
        cc.valid = true;
        cc.plan = frames[0].plan;
        cc.flags = flags;
        cc.rf = rf_dev;
        cc.out = out_dev;
        cc.ns = n_samples;
        cc.na = n_angles;
        cc.pdas_p = h->pdas_p;
        cc.stream = h->stream;
        cc.frames = frames;
        cc.hl = std::move(hl);
    }
    return rc;
}

// Plane-wave f-k migration of one device-resident frame onto the native grid
// (one column per element, depth step c / (2 fs)).
BF_API int bf_fkmig(bf_handle *h, const int16_t *rf_dev, int32_t n_samples,
                    const double *angles_rad, int32_t n_angles, uint32_t flags, float *out_dev)
{
    if (!h)
        return fail(BF_EINVAL, "null handle");
    if (!rf_dev || !out_dev || !angles_rad)
        return fail(BF_EINVAL, "null argument");
    if (flags & ~((uint32_t)BF_OUT_MASK | (uint32_t)BF_FK_STOLT))
        return fail(BF_EINVAL, "bf_fkmig takes only an output stage and BF_FK_STOLT in its flags");
    const bool stolt = (flags & BF_FK_STOLT) != 0;
    const int stage = flags & BF_OUT_MASK;
    if (stage != BF_OUT_RF && stage != BF_OUT_ENV && stage != BF_OUT_LOGDB)
        return fail(BF_EINVAL, "unknown output stage bits");
    if (n_samples < 2 || n_samples > 4096)
        return fail(BF_EINVAL, "bf_fkmig handles 2 <= n_samples <= 4096 (got %d)", n_samples);
    if (n_angles < 1 || n_angles > 256)
        return fail(BF_EINVAL, "n_angles must be in [1, 256], got %d", n_angles);
    for (int a = 0; a < n_angles; ++a)
        if (!std::isfinite(angles_rad[a]) || std::fabs(angles_rad[a]) >= 1.5707963267948966)
            return fail(BF_EINVAL, "angle %d (%g rad) outside (-pi/2, pi/2)", a, angles_rad[a]);
    const int ne = h->g.ne;
    if (ne < 2 || ne > 2048)
        return fail(BF_EINVAL, "bf_fkmig needs 2 to 2048 elements (got %d)", ne);
    const double pitch = (h->g.xe[ne - 1] - h->g.xe[0]) / (double)(ne - 1);
    for (int i = 0; i < ne; ++i)
        if (std::fabs(h->g.xe[i] - (h->g.xe[0] + i * pitch)) > 1e-9 * std::fabs(pitch) * ne)
            return fail(BF_EINVAL, "bf_fkmig needs equally spaced elements");
    cudaSetDevice(h->device);
    if (!is_device_pointer(rf_dev) || !is_device_pointer(out_dev))
        return fail(BF_EINVAL, "bf_fkmig needs device pointers");
    int nt = 1, lgt = 0, nk = 1, lgk = 0;
    while (nt < 2 * n_samples) {
        nt <<= 1;
        ++lgt;
    }
    while (nk < 2 * ne) {
        nk <<= 1;
        ++lgk;
    }
    const double c = h->g.c, fs = h->g.fs, dz = c / (2.0 * fs);
    std::vector<float> beta((size_t)n_angles * ne);
    std::vector<double> sc((size_t)2 * n_angles);
    for (int a = 0; a < n_angles; ++a) {
        sc[2 * a] = std::sin(angles_rad[a]);
        sc[2 * a + 1] = std::cos(angles_rad[a]);
        for (int i = 0; i < ne; ++i) {
            const double x = ((double)i - 0.5 * (double)(ne - 1)) * pitch;
            beta[(size_t)a * ne + i] = (float)(kPi * x * sc[2 * a] / ((double)nt * dz));
        }
    }
    // The mapping tables (geometry only): rebuilt when the sample count, the
    // angles or the mapping change.
    const int half = nt / 2;
    const size_t npts = (size_t)half * nk;
    std::vector<double> key{(double)n_samples, stolt ? 1.0 : 0.0};
    key.insert(key.end(), angles_rad, angles_rad + n_angles);
    const bool rebuild = key != h->fk_key;
    std::shared_ptr<EnvTablesDev> tt, tk;
    int rc = env_tables(nt, tt);
    if (!rc)
        rc = env_tables(nk, tk);
    const size_t nf = (size_t)nt / 2 + 1, img = (size_t)ne * n_samples;
    if (!rc)
        rc = h->fk_D.ensure((size_t)n_angles * nf * nk * sizeof(float2));
    if (!rc)
        rc = h->fk_spec.ensure((size_t)(nt / 2) * nk * sizeof(float2));
    if (!rc && stage == BF_OUT_LOGDB)
        rc = h->fk_img.ensure(img * sizeof(float));
    if (!rc)
        rc = h->fk_max.ensure(sizeof(unsigned));
    if (!rc)
        rc = h->fk_beta.ensure(beta.size() * sizeof(float));
    if (!rc && rebuild)
        rc = h->fk_i0.ensure((size_t)n_angles * npts * sizeof(int));
    if (!rc && rebuild)
        rc = h->fk_aw.ensure((size_t)n_angles * npts * sizeof(float2));
    if (rc)
        return rc;
    if (rebuild) {
        std::vector<int> i0;
        std::vector<float> aw;
        fk_mapping_tables(ne, nt, nk, pitch, dz, sc, stolt, i0, aw);
        cudaError_t ce = cudaMemcpy(h->fk_i0.p, i0.data(), i0.size() * sizeof(int),
                                    cudaMemcpyHostToDevice);
        if (ce == cudaSuccess)
            ce = cudaMemcpy(h->fk_aw.p, aw.data(), aw.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (ce != cudaSuccess)
            return cuda_fail(ce, "bf_fkmig mapping tables");
        h->fk_key = key;
    }
    h->call.clear();  // the device tables above may have moved
    cudaStream_t st = h->stream;
    cudaError_t e = cudaMemcpyAsync(h->fk_beta.p, beta.data(), beta.size() * sizeof(float),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && stage == BF_OUT_LOGDB)
        e = cudaMemsetAsync(h->fk_max.p, 0, sizeof(unsigned), st);
    if (e != cudaSuccess)
        return cuda_fail(e, "bf_fkmig setup");
    FkJob J{};
    J.rf = rf_dev;
    J.D = (float2 *)h->fk_D.p;
    J.spec = (float2 *)h->fk_spec.p;
    J.img = stage == BF_OUT_LOGDB ? (float *)h->fk_img.p : out_dev;
    J.maxbits = stage == BF_OUT_LOGDB ? (unsigned *)h->fk_max.p : nullptr;
    J.beta = (const float *)h->fk_beta.p;
    J.map_i0 = (const int *)h->fk_i0.p;
    J.map_aw = (const float2 *)h->fk_aw.p;
    J.tw_t = (const float2 *)tt->tw.p;
    J.tw_k = (const float2 *)tk->tw.p;
    J.na = n_angles;
    J.ne = ne;
    J.ns = n_samples;
    J.nt = nt;
    J.lgt = lgt;
    J.nk = nk;
    J.lgk = lgk;
    e = launch_fkmig(J, st);
    if (e != cudaSuccess)
        return cuda_fail(e, "f-k migration launch");
    if (stage == BF_OUT_LOGDB) {
        // the log stage of the beamformer, one job over the native image
        LogJob l{};
        l.env = J.img;
        l.out = out_dev;
        l.maxbits = J.maxbits;
        l.n = (int)img;
        l.vec4 = (img % 4 == 0 && ((uintptr_t)l.env & 15) == 0 && ((uintptr_t)l.out & 15) == 0) ? 1 : 0;
        rc = h->fk_log.upload(&l, sizeof l);
        int zero = 0;
        if (!rc)
            rc = h->fk_logp.upload(&zero, sizeof zero);
        if (rc)
            return rc;
        e = launch_log((const LogJob *)h->fk_log.p, (const int *)h->fk_logp.p, 1,
                       log_blocks((long long)img), 70.0f, st);
        if (e != cudaSuccess)
            return cuda_fail(e, "log launch");
    }
    return BF_OK;
}

BF_API int bf_beamform_plain(bf_handle *h, const int16_t *rf_dev, int32_t n_samples,
                             const double *angles_rad, int32_t n_angles, uint32_t flags,
                             float *out_dev)
{
    if (!h)
        return fail(BF_EINVAL, "null handle");
    if (!rf_dev || !out_dev)
        return fail(BF_EINVAL, "null data pointer");
    if (flags & BF_PREC_MASK)
        return fail(BF_EINVAL, "the plain kernel computes from int16 records in FP32 only");
    if (flags & BF_IQ_MASK)
        return fail(BF_EINVAL, "the plain kernel computes the RF combiners only");
    cudaSetDevice(h->device);
    if (!is_device_pointer(rf_dev) || !is_device_pointer(out_dev))
        return fail(BF_EINVAL, "bf_beamform_plain needs device pointers");
    h->call.clear();  // the plain path reuses the handle's scratch
    std::vector<FramePrep> frames(1);
    int rc = prepare_frame(h, rf_dev, n_samples, angles_rad, n_angles, flags, out_dev, h->scratch,
                           frames[0]);
    if (rc)
        return rc;
    HostLaunch hl;
    build_launch(frames, hl);
    const BfJob &job = hl.jobs[0];
    cudaError_t e = launch_plain(job, rf_dev, (const int2 *)frames[0].plan->valid.p,
                                 (const float *)h->dx2.p, pad_cols(h->g.nx), n_samples, h->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "plain kernel launch");
    if (frames[0].stage == BF_OUT_RF)
        return BF_OK;
    // envelope / log stages as in bf_beamform
    hl.jobs.clear();
    hl.groups.clear();
    hl.igroups.clear();
    rc = h->launch.upload(hl, h->stream, true);
    if (!rc && !h->err_cleared) {
        cudaMemsetAsync(h->launch.err.p, 0, sizeof(int), h->stream);
        h->err_cleared = true;
    }
    if (!rc)
        rc = cudaMemsetAsync(frames[0].maxbits, 0, 4 * sizeof(unsigned), h->stream) == cudaSuccess
                 ? BF_OK
                 : fail(BF_ECUDA, "cudaMemsetAsync");
    if (!rc && !hl.env.empty()) {
        e = launch_envelope((const EnvJob *)h->launch.env.p, (const int *)h->launch.env_prefix.p,
                            (int)hl.env.size(), hl.env_blocks, hl.env_smem, h->stream);
        if (e != cudaSuccess)
            rc = cuda_fail(e, "envelope launch");
    }
    if (!rc && !hl.envw.empty()) {
        e = launch_envelope_warp((const EnvJob *)h->launch.envw.p,
                                 (const int *)h->launch.envw_prefix.p, (int)hl.envw.size(),
                                 hl.envw_pairs, h->stream);
        if (e != cudaSuccess)
            rc = cuda_fail(e, "envelope launch");
    }
    if (!rc && !hl.log.empty()) {
        e = launch_log((const LogJob *)h->launch.log.p, (const int *)h->launch.blk_prefix.p,
                       (int)hl.log.size(), hl.log_blocks, 70.0f, h->stream);
        if (e != cudaSuccess)
            rc = cuda_fail(e, "log launch");
    }
    return rc;
}

BF_API int bf_sync(bf_handle *h)
{
    if (!h)
        return fail(BF_EINVAL, "null handle");
    cudaSetDevice(h->device);
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamSynchronize");
    if (!h->launch.err.p)
        return BF_OK;
    return read_device_error(h->launch, h->stream);
}

// Host-only view of the decision tables (no CUDA involved): first / last
// counted row per (angle, column, channel) and aperture counts per pixel.
BF_API int bf_host_tables(const bf_geometry *geom, const bf_grid *grid, double fs_hz, double f0_hz,
                          double c_mps, int32_t n_samples, const double *angles_rad,
                          int32_t n_angles, int32_t *valid_rows, uint16_t *aperture_count)
{
    if (!geom || !grid || !angles_rad || n_angles < 1 || n_samples < 2)
        return fail(BF_EINVAL, "bad arguments");
    GeomHost g;
    g.ne = geom->n_elements;
    if (g.ne < 1 || grid->nx < 1 || grid->nz < 1 || !(geom->f_number > 0.0))
        return fail(BF_EINVAL, "bad geometry");
    g.xe.resize(g.ne);
    for (int i = 0; i < g.ne; ++i)
        g.xe[i] = geom->x_elem_m ? geom->x_elem_m[i]
                                 : ((double)i - 0.5 * (double)(g.ne - 1)) * geom->pitch_m;
    g.fnum = geom->f_number;
    g.nx = grid->nx;
    g.nz = grid->nz;
    g.x0 = grid->x0_m;
    g.x1 = grid->x1_m;
    g.z0 = grid->z0_m;
    g.z1 = grid->z1_m;
    g.fs = fs_hz;
    g.f0 = f0_hz;
    g.c = c_mps;
    GeometryHost geo;
    geometry_tables(g, geo);
    PlanHost ph;
    angle_tables(g, geo, n_samples, std::vector<double>(angles_rad, angles_rad + n_angles),
                 kPrecF32, 8, kTileConfigs[0].stage_bytes, ph);
    const int nxp = pad_cols(g.nx);
    if (valid_rows)  // [na][ne][nxp][2] -> [na][nx][ne][2]
        for (int a = 0; a < n_angles; ++a)
            for (int ix = 0; ix < g.nx; ++ix)
                for (int i = 0; i < g.ne; ++i)
                    for (int q = 0; q < 2; ++q)
                        valid_rows[(((size_t)a * g.nx + ix) * g.ne + i) * 2 + q] =
                            ph.valid[(((size_t)a * g.ne + i) * nxp + ix) * 2 + q];
    if (aperture_count)
        std::memcpy(aperture_count, geo.apcnt.data(), geo.apcnt.size() * sizeof(uint16_t));
    return BF_OK;
}

// Plan introspection: tile shape and window sizes of the plan a frame with
// these arguments uses (built if needed), and optionally its window table.
BF_API int bf_plan_info(bf_handle *h, int32_t n_samples, const double *angles_rad,
                        int32_t n_angles, uint32_t flags, int32_t *info8, int32_t *wtab,
                        size_t wtab_entries)
{
    int rc = check_frame_args(h, n_samples, angles_rad, n_angles, flags);
    if (rc)
        return rc;
    if (!info8)
        return fail(BF_EINVAL, "null info");
    cudaSetDevice(h->device);
    Plan *p = nullptr;
    rc = handle_plan(h, n_samples, angles_rad, n_angles, flags, &p);
    if (rc)
        return rc;
    const size_t n = (size_t)n_angles * p->tiles_x * p->tiles_z * h->g.ne;
    const int32_t v[8] = {p->wmax, p->box, p->group, p->rows, p->tiles_x, p->tiles_z, p->nsp,
                          (int32_t)n};
    std::memcpy(info8, v, sizeof v);
    if (wtab) {
        if (wtab_entries < n)
            return fail(BF_EINVAL, "window table needs %zu entries", n);
        cudaError_t e = cudaMemcpy(wtab, p->wtab.p, n * sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaMemcpy (window table)");
    }
    return BF_OK;
}

// Autotuner: times the beamforming launches of `frames` copies of this
// workload under every tile configuration (synthetic zero records: the work
// does not depend on the data) and keeps the fastest for the handle's later
// work on it.
BF_API int bf_autotune(bf_handle *h, int32_t n_samples, const double *angles_rad,
                       int32_t n_angles, uint32_t flags, int32_t frames, int32_t *rows_out,
                       int32_t *stage_bytes_out, float *candidate_us, int32_t n_candidates)
{
    int rc = check_frame_args(h, n_samples, angles_rad, n_angles, flags);
    if (rc)
        return rc;
    if (frames < 1 || frames > 256)
        return fail(BF_EINVAL, "frames must be in [1, 256], got %d", frames);
    cudaSetDevice(h->device);
    const uint32_t fl = flags & ~(uint32_t)BF_OUT_MASK;  // beamformed output only
    const size_t rf_bytes = (size_t)n_angles * h->g.ne * n_samples * sizeof(int16_t);
    const size_t out_bytes = frame_out_bytes(h, fl);
    DevMem rf, out;
    rc = rf.ensure(rf_bytes);
    if (!rc)
        rc = out.ensure(out_bytes * frames);
    if (rc)
        return rc;
    cudaStream_t st;
    cudaError_t e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    cudaEvent_t marks[4] = {};
    for (auto &m : marks)
        if (e == cudaSuccess)
            e = cudaEventCreate(&m);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(rf.p, 0, rf_bytes, st);
    std::vector<FrameScratch> scratch(frames);
    std::vector<float> best_us(kNumTileConfigs, -1.f);
    int best = -1;
    for (int c = 0; c < kNumTileConfigs && e == cudaSuccess && !rc; ++c) {
        std::vector<FramePrep> fr(frames);
        int prc = BF_OK;
        for (int i = 0; i < frames && !prc; ++i)
            prc = prepare_frame(h, (const int16_t *)rf.p, n_samples, angles_rad, n_angles, fl,
                                (float *)out.p + (size_t)i * (out_bytes / sizeof(float)),
                                scratch[i], fr[i], c, kMaxFramesPerJob);
        if (prc)
            continue;  // this configuration does not fit the workload
        HostLaunch hl;
        build_launch(fr, hl);
        DeviceLaunch dl;
        rc = upload_maps(fr, st, false);
        if (!rc)
            rc = dl.upload(hl, st, false);
        if (!rc && cudaMemsetAsync(dl.err.p, 0, sizeof(int), st) != cudaSuccess)
            rc = fail(BF_ECUDA, "cudaMemsetAsync");
        std::vector<float> t;
        for (int rep = 0; rep < 4 && !rc; ++rep) {  // one warm-up, three timed
            rc = enqueue(fr, hl, dl, st, marks);
            if (!rc && cudaStreamSynchronize(st) != cudaSuccess)
                rc = fail(BF_ECUDA, "autotune replay");
            float ms = 0.f;
            if (!rc && cudaEventElapsedTime(&ms, marks[1], marks[2]) == cudaSuccess && rep > 0)
                t.push_back(ms * 1e3f);
        }
        if (!rc)
            rc = read_device_error(dl, st);
        if (rc || t.empty())
            break;
        std::sort(t.begin(), t.end());
        best_us[c] = t[t.size() / 2];
        if (best < 0 || best_us[c] < best_us[best])
            best = c;
    }
    for (auto &m : marks)
        if (m)
            cudaEventDestroy(m);
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
    if (rc)
        return rc;
    if (e != cudaSuccess)
        return cuda_fail(e, "autotune setup");
    if (best < 0)
        return fail(BF_EINVAL, "no tile configuration fits this workload");
    {
        std::lock_guard<std::mutex> lk(h->mu);
        PlanKey key{n_samples, frame_prec(flags),
                    std::vector<double>(angles_rad, angles_rad + n_angles), 0};
        h->tuned[key] = best;
    }
    if (rows_out)
        *rows_out = kTileConfigs[best].rows;
    if (stage_bytes_out)
        *stage_bytes_out = kTileConfigs[best].stage_bytes;
    if (candidate_us)
        for (int c = 0; c < std::min<int>(n_candidates, kNumTileConfigs); ++c)
            candidate_us[c] = best_us[c];
    return BF_OK;
}

// ------------------------------------------------------------------ batch --

BF_API int bf_batch_create(const bf_frame *frames, int32_t n, bf_batch **out)
{
    if (!frames || !out || n < 1)
        return fail(BF_EINVAL, "bad batch arguments");
    *out = nullptr;
    auto b = std::make_unique<bf_batch>();
    b->scratch.resize(n);
    b->frames.resize(n);
    int dev = -1;
    for (int i = 0; i < n; ++i) {
        const bf_frame &f = frames[i];
        if (!f.h || !f.rf_dev || !f.out_dev)
            return fail(BF_EINVAL, "frame %d: null handle or data pointer", i);
        if (dev < 0)
            dev = f.h->device;
        else if (dev != f.h->device)
            return fail(BF_EINVAL, "frame %d: all frames of a batch must use one device", i);
        cudaSetDevice(dev);
        if (!is_device_pointer(f.rf_dev) || !is_device_pointer(f.out_dev))
            return fail(BF_EINVAL, "frame %d: batches need device pointers", i);
        int rc = prepare_frame(f.h, f.rf_dev, f.n_samples, f.angles_rad, f.n_angles,
                               f.mode_and_flags, f.out_dev, b->scratch[i], b->frames[i], -1,
                               kMaxFramesPerJob);
        if (rc)
            return fail(rc, "frame %d: %s", i, g_err.c_str());
    }
    b->device = dev;
    build_launch(b->frames, b->hl);
    int rc = upload_maps(b->frames, nullptr, false);
    if (!rc)
        rc = b->dl.upload(b->hl, nullptr, false);
    if (rc)
        return rc;
    cudaMemset(b->dl.err.p, 0, sizeof(int));
    // Capture the batch's launches once; bf_batch_launch replays the graph.
    // The stage marks sit on a side branch of the graph (MarkBranch).
    cudaStream_t cap;
    cudaError_t e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
    if (e != cudaSuccess)
        return cuda_fail(e, "cudaStreamCreate");
    MarkBranch br;
    e = cudaStreamCreateWithFlags(&br.side, cudaStreamNonBlocking);
    for (auto &f : br.fork)
        if (e == cudaSuccess)
            e = cudaEventCreateWithFlags(&f, cudaEventDisableTiming);
    if (e == cudaSuccess)
        e = cudaEventCreateWithFlags(&br.join, cudaEventDisableTiming);
    for (auto &m : b->marks)
        if (e == cudaSuccess)
            e = cudaEventCreate(&m);
    b->launches = (int)b->hl.igroups.size() + (b->hl.demod.empty() ? 0 : 1) +
                  (int)b->hl.groups.size() + (b->hl.env.empty() ? 0 : 1) + (b->hl.envw.empty() ? 0 : 1) +
                  (b->hl.log.empty() ? 0 : 1);
    if (e == cudaSuccess)
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = enqueue(b->frames, b->hl, b->dl, cap, b->marks, &br);
        cudaGraph_t g = nullptr;
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (!rc && e2 == cudaSuccess) {
            e2 = cudaGraphInstantiate(&b->exec, g, 0);
            if (e2 != cudaSuccess)
                rc = cuda_fail(e2, "cudaGraphInstantiate");
        } else if (!rc) {
            rc = cuda_fail(e2, "cudaStreamEndCapture");
        }
        if (g)
            cudaGraphDestroy(g);
    } else {
        rc = cuda_fail(e, "cudaStreamBeginCapture");
    }
    cudaStreamDestroy(cap);
    for (auto &f : br.fork)
        if (f)
            cudaEventDestroy(f);
    if (br.join)
        cudaEventDestroy(br.join);
    if (br.side)
        cudaStreamDestroy(br.side);
    if (rc)
        return rc;
    *out = b.release();
    return BF_OK;
}

BF_API int bf_batch_launch(bf_batch *b, void *stream)
{
    if (!b)
        return fail(BF_EINVAL, "null batch");
    cudaSetDevice(b->device);
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    return e == cudaSuccess ? BF_OK : cuda_fail(e, "cudaGraphLaunch");
}

BF_API int bf_batch_status(bf_batch *b, void *stream)
{
    if (!b)
        return fail(BF_EINVAL, "null batch");
    cudaSetDevice(b->device);
    return read_device_error(b->dl, (cudaStream_t)stream);
}

BF_API int bf_batch_timing(bf_batch *b, float *ms3, int32_t *kernel_launches)
{
    if (!b || !ms3)
        return fail(BF_EINVAL, "null argument");
    cudaSetDevice(b->device);
    for (int k = 0; k < 3; ++k) {
        cudaError_t e = cudaEventElapsedTime(&ms3[k], b->marks[k], b->marks[k + 1]);
        if (e != cudaSuccess)
            return cuda_fail(e, "cudaEventElapsedTime");
    }
    if (kernel_launches)
        *kernel_launches = b->launches;
    return BF_OK;
}

BF_API int bf_batch_destroy(bf_batch *b)
{
    if (!b)
        return fail(BF_EINVAL, "null batch");
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    if (b->exec)
        cudaGraphExecDestroy(b->exec);
    for (auto &m : b->marks)
        if (m)
            cudaEventDestroy(m);
    delete b;
    return BF_OK;
}

}  // extern "C"
