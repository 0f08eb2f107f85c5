// runtime.cu -- error state, launch counter, device properties and the
// per-(device, stream) scratch cache of the accr library.
#include <math.h>
#include <stdarg.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "common.cuh"
#include "debug.cuh"

namespace accr {

static thread_local std::string t_last_error;
static std::atomic<uint64_t> g_launches{0};

int log_level() {
    static const int level = [] {
        const char *e = getenv("ACCR_LOG");
        return e ? atoi(e) : 0;
    }();
    return level;
}

void log_msg(int level, const char *fmt, ...) {
    if (log_level() < level) return;
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    fprintf(stderr, "accr: %s\n", buf);
}

TraceRange::TraceRange(const char *name) { nvtxRangePushA(name); }
TraceRange::~TraceRange() { nvtxRangePop(); }

int set_error(int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    t_last_error = buf;
    if (log_level() >= 1) fprintf(stderr, "accr: error %d: %s\n", code, buf);
    return code;
}

void clear_error() { t_last_error.clear(); }

int cuda_check(cudaError_t e, const char *where) {
    if (e == cudaSuccess) return ACCR_OK;
    return set_error(ACCR_ECUDA, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

static std::atomic<int64_t> g_faults[4];

bool fault_take(int kind) {
    if (kind < 1 || kind > 3) return false;
    int64_t v = g_faults[kind].load(std::memory_order_relaxed);
    while (v > 0) {
        if (g_faults[kind].compare_exchange_weak(v, v - 1)) return true;
    }
    return false;
}

int launch_guard(const char *what) {
    if (fault_take(ACCR_FAULT_LAUNCH)) return set_error(ACCR_ECUDA, "%s: injected launch failure", what);
    return ACCR_OK;
}

int launched(const char *what, int kernels) {
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(e, what);
    g_launches.fetch_add((uint64_t)kernels, std::memory_order_relaxed);
    return ACCR_OK;
}

// ---- device properties ------------------------------------------------------
static std::mutex g_dev_mu;
static std::map<int, DeviceInfo> g_dev;

const DeviceInfo &device_info() {
    int dev = 0;
    cudaGetDevice(&dev);
    // per-thread memo of the last device (map entries never move): no lock on
    // the launch path of a thread that keeps to one device
    static thread_local int t_dev = -1;
    static thread_local const DeviceInfo *t_info = nullptr;
    if (dev == t_dev) return *t_info;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    auto hit = g_dev.find(dev);
    if (hit != g_dev.end()) {
        t_dev = dev;
        t_info = &hit->second;
        return hit->second;
    }
    DeviceInfo d{};
    d.id = dev;
    cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&d.l2_bytes, cudaDevAttrL2CacheSize, dev);
    cudaDeviceGetAttribute(&d.max_smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (d.sms <= 0) d.sms = 1;
    const DeviceInfo &ref = g_dev.emplace(dev, d).first->second;
    t_dev = dev;
    t_info = &ref;
    return ref;
}

// ---- scratch -----------------------------------------------------------------
struct ScratchEntry {
    Scratch s{};
    void *host = nullptr;
    size_t host_bytes = 0;
    unsigned *zw = nullptr;  // zeroed_words_for
    size_t zw_n = 0;
    std::atomic<uint64_t> gen{0};     // bumped whenever `s` is replaced
    std::atomic<uint64_t> zw_gen{0};  // bumped whenever `zw` is replaced
};
static std::mutex g_scr_mu;
static std::map<std::pair<int, uintptr_t>, ScratchEntry *> g_scr;

static ScratchEntry *entry_for(accr_stream_t stream) {
    int dev = 0;
    cudaGetDevice(&dev);
    auto key = std::make_pair(dev, (uintptr_t)stream);
    auto it = g_scr.find(key);
    if (it != g_scr.end()) return it->second;
    ScratchEntry *e = new ScratchEntry();
    g_scr.emplace(key, e);
    return e;
}

// Per-thread memo of the last (device, stream) scratch: a repeated call on the
// same stream takes no lock unless the scratch was replaced meanwhile.
struct ScratchMemo {
    int dev = -1;
    accr_stream_t stream = nullptr;
    ScratchEntry *e = nullptr;
    uint64_t gen = 0;
    size_t bytes = 0;
};
static thread_local ScratchMemo t_scr;

Scratch *scratch_for(accr_stream_t stream, size_t bytes) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (t_scr.e && t_scr.dev == dev && t_scr.stream == stream && bytes <= t_scr.bytes &&
        t_scr.e->gen.load(std::memory_order_acquire) == t_scr.gen)
        return &t_scr.e->s;
    std::lock_guard<std::mutex> lk(g_scr_mu);
    ScratchEntry *e = entry_for(stream);
    auto remember = [&] {
        t_scr.dev = dev;
        t_scr.stream = stream;
        t_scr.e = e;
        t_scr.gen = e->gen.load(std::memory_order_relaxed);
        t_scr.bytes = e->s.bytes;
        return &e->s;
    };
    if (e->s.counters && e->s.bytes >= bytes) return remember();
    if (fault_take(ACCR_FAULT_ALLOC)) {
        set_error(ACCR_ENOMEM, "scratch: injected allocation failure");
        return nullptr;
    }
    // first use, or growth: the old buffer may still be read by work queued on
    // this stream, so drain the stream before releasing it
    if (e->s.counters) {
        if (cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "scratch grow") != ACCR_OK)
            return nullptr;
        cudaFree(e->s.counters);
        e->s = Scratch{};
        e->gen.fetch_add(1, std::memory_order_release);
    }
    size_t want = bytes < (1u << 20) ? (1u << 20) : bytes;
    want = (want + 4095) & ~(size_t)4095;
    const size_t head = 256;  // counters
    void *p = nullptr;
    if (cudaMalloc(&p, head + want) != cudaSuccess) {
        cudaGetLastError();
        set_error(ACCR_ENOMEM, "scratch: cudaMalloc of %zu bytes failed", head + want);
        return nullptr;
    }
    if (cuda_check(cudaMemset(p, 0, head), "scratch clear") != ACCR_OK) {
        cudaFree(p);
        return nullptr;
    }
    e->s.counters = (unsigned *)p;
    e->s.buf = (char *)p + head;
    e->s.bytes = want;
    e->gen.fetch_add(1, std::memory_order_release);
    return remember();
}

void *host_staging_for(accr_stream_t stream, size_t bytes) {
    std::lock_guard<std::mutex> lk(g_scr_mu);
    ScratchEntry *e = entry_for(stream);
    if (e->host && e->host_bytes >= bytes) return e->host;
    if (fault_take(ACCR_FAULT_ALLOC)) {
        set_error(ACCR_ENOMEM, "host staging: injected allocation failure");
        return nullptr;
    }
    if (e->host) {
        cudaStreamSynchronize((cudaStream_t)stream);
        cudaFreeHost(e->host);
        e->host = nullptr;
    }
    size_t want = bytes < 65536 ? 65536 : bytes;
    if (cudaMallocHost(&e->host, want) != cudaSuccess) {
        cudaGetLastError();
        e->host = nullptr;
        set_error(ACCR_ENOMEM, "host staging: cudaMallocHost of %zu bytes failed", want);
        return nullptr;
    }
    e->host_bytes = want;
    return e->host;
}

// Per-thread memo of the last (device, stream) zeroed words, as for scratch.
struct ZeroedMemo {
    int dev = -1;
    accr_stream_t stream = nullptr;
    ScratchEntry *e = nullptr;
    uint64_t gen = 0;
    size_t n = 0;
    unsigned *zw = nullptr;
};
static thread_local ZeroedMemo t_zw;

unsigned *zeroed_words_for(accr_stream_t stream, size_t n) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (t_zw.e && t_zw.dev == dev && t_zw.stream == stream && n <= t_zw.n &&
        t_zw.e->zw_gen.load(std::memory_order_acquire) == t_zw.gen)
        return t_zw.zw;
    std::lock_guard<std::mutex> lk(g_scr_mu);
    ScratchEntry *e = entry_for(stream);
    auto remember = [&] {
        t_zw.dev = dev;
        t_zw.stream = stream;
        t_zw.e = e;
        t_zw.gen = e->zw_gen.load(std::memory_order_relaxed);
        t_zw.n = e->zw_n;
        t_zw.zw = e->zw;
        return e->zw;
    };
    if (e->zw && e->zw_n >= n) return remember();
    if (fault_take(ACCR_FAULT_ALLOC)) {
        set_error(ACCR_ENOMEM, "zeroed words: injected allocation failure");
        return nullptr;
    }
    if (e->zw) {  // work queued on this stream may still use the old words
        if (cuda_check(cudaStreamSynchronize((cudaStream_t)stream), "zeroed words grow") != ACCR_OK) return nullptr;
        cudaFree(e->zw);
        e->zw = nullptr;
        e->zw_n = 0;
        e->zw_gen.fetch_add(1, std::memory_order_release);
    }
    size_t want = n < 4096 ? 4096 : n;
    if (cudaMalloc((void **)&e->zw, want * sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        e->zw = nullptr;
        set_error(ACCR_ENOMEM, "zeroed words: cudaMalloc of %zu words failed", want);
        return nullptr;
    }
    if (cuda_check(cudaMemsetAsync(e->zw, 0, want * sizeof(unsigned), (cudaStream_t)stream), "zeroed words clear") !=
        ACCR_OK) {
        cudaFree(e->zw);
        e->zw = nullptr;
        return nullptr;
    }
    e->zw_n = want;
    e->zw_gen.fetch_add(1, std::memory_order_release);
    return remember();
}

}  // namespace accr

extern "C" ACCR_API const char *accr_last_error(void) { return accr::t_last_error.c_str(); }

extern "C" ACCR_API uint64_t accr_launch_count(void) {
    return accr::g_launches.load(std::memory_order_relaxed);
}

extern "C" ACCR_API int32_t accr_version(void) { return ACCR_VERSION; }

// ---- debug builds: readers of the translation units' status words -----------------
namespace accr {
static std::vector<DebugReader> &debug_readers() {
    static std::vector<DebugReader> *v = new std::vector<DebugReader>();  // filled during static init
    return *v;
}
void debug_register(DebugReader reader) { debug_readers().push_back(reader); }
}  // namespace accr

extern "C" ACCR_API int accr_debug_report(uint64_t *violations, uint32_t *first_site, int32_t *checked,
                                          int32_t clear) {
    accr::clear_error();
    if (!violations || !first_site || !checked) return accr::set_error(ACCR_EINVAL, "accr_debug_report: NULL argument");
    *violations = 0;
    *first_site = 0;
#ifdef ACCR_DEBUG
    *checked = 1;
#else
    *checked = 0;
#endif
    for (accr::DebugReader r : accr::debug_readers()) {
        unsigned long long n = 0, site = 0;
        if (r(&n, &site, clear != 0) != ACCR_OK)
            return accr::set_error(ACCR_ECUDA, "accr_debug_report: reading a status word failed");
        *violations += n;
        if (!*first_site && site) *first_site = (uint32_t)site;
    }
    return ACCR_OK;
}

extern "C" ACCR_API int accr_fault_inject(int32_t kind, int64_t count) {
    accr::clear_error();
    if (kind < 1 || kind > 3 || count < 0) return accr::set_error(ACCR_EINVAL, "accr_fault_inject: bad kind or count");
    accr::g_faults[kind].store(count);
    return ACCR_OK;
}

// ---- clause lowering -----------------------------------------------------------
#include "fold.cuh"

namespace accr {

static const char *op_name(int op) {
    static const char *names[] = {"+", "*", "max", "min", "&", "|", "^", "&&", "||"};
    return (op >= 0 && op <= 8) ? names[op] : "?";
}

// OpenACC identity of the operator in the variable's type (bits).
static uint64_t var_identity(int op, int acc) {
    const bool i64 = acc == ACCR_I64;
    switch (acc) {
    case ACCR_I32:
    case ACCR_I64: {
        int64_t v = 0;
        switch (op) {
        case ACCR_ADD: v = 0; break;
        case ACCR_MUL: v = 1; break;
        case ACCR_MAX: v = i64 ? INT64_MIN : INT32_MIN; break;
        case ACCR_MIN: v = i64 ? INT64_MAX : INT32_MAX; break;
        case ACCR_BAND: v = -1; break;
        case ACCR_LAND: v = 1; break;
        default: v = 0; break;
        }
        return i64 ? (uint64_t)v : (uint64_t)(uint32_t)(int32_t)v;
    }
    case ACCR_F32: {
        float f = op == ACCR_MUL ? 1.0f : op == ACCR_MAX ? -INFINITY : op == ACCR_MIN ? INFINITY : 0.0f;
        return f2u(f);
    }
    default: {
        double d = op == ACCR_MUL ? 1.0 : op == ACCR_MAX ? -INFINITY : op == ACCR_MIN ? INFINITY : 0.0;
        return d2u(d);
    }
    }
}

int lower_clauses(int in_type, const accr_clause *c, int nc, unsigned flags, ClauseDev *dev) {
    if (!type_valid(in_type)) return set_error(ACCR_EINVAL, "element type %d is not an accr_type", in_type);
    if (nc < 1 || nc > ACCR_MAX_CLAUSES)
        return set_error(ACCR_EINVAL, "nclauses = %d (must be 1..%d)", nc, ACCR_MAX_CLAUSES);
    if (!c) return set_error(ACCR_EINVAL, "clauses is NULL");
    const bool e64 = type_bytes(in_type) == 8;
    for (int k = 0; k < nc; ++k) {
        const int op = c[k].op, acc = c[k].acc_type;
        if (op < ACCR_ADD || op > ACCR_LOR) return set_error(ACCR_EINVAL, "clause %d: operator %d is not an accr_op", k, op);
        if (!type_valid(acc)) return set_error(ACCR_EINVAL, "clause %d: variable type %d is not an accr_type", k, acc);
        if (type_is_int(in_type) != type_is_int(acc))
            return set_error(ACCR_ETYPE, "clause %d: %s elements into a %s variable", k,
                             type_is_int(in_type) ? "integer" : "floating-point",
                             type_is_int(acc) ? "integer" : "floating-point");
        if (type_bytes(acc) < type_bytes(in_type))
            return set_error(ACCR_ETYPE, "clause %d: variable narrower than the elements", k);
        if (!type_is_int(acc) && op >= ACCR_BAND)
            return set_error(ACCR_ETYPE, "clause %d: operator %s is not defined on floating point", k, op_name(op));
        if (!c[k].out) return set_error(ACCR_EINVAL, "clause %d: out is NULL", k);
        ClauseDev &d = dev[k];
        memset(&d, 0, sizeof d);
        d.op = op;
        d.acc_type = acc;
        d.out = c[k].out;
        const bool a64 = type_bytes(acc) == 8;
        if (type_is_int(acc)) {
            switch (op) {
            case ACCR_ADD: d.wcode = a64 ? W_ADD64 : W_ADD32; d.ident = 0; break;
            case ACCR_MUL: d.wcode = a64 ? W_MUL64 : W_MUL32; d.ident = 1; break;
            case ACCR_MAX: d.wcode = W_MAXI; d.ident = e64 ? (uint64_t)INT64_MIN : (uint64_t)(uint32_t)INT32_MIN; break;
            case ACCR_MIN: d.wcode = W_MINI; d.ident = e64 ? (uint64_t)INT64_MAX : (uint64_t)(uint32_t)INT32_MAX; break;
            case ACCR_BAND: d.wcode = W_AND; d.ident = e64 ? ~0ull : 0xffffffffull; break;
            case ACCR_BOR: d.wcode = W_OR; d.ident = 0; break;
            case ACCR_BXOR: d.wcode = W_XOR; d.ident = 0; break;
            case ACCR_LAND: d.wcode = W_LAND; d.ident = 1; break;
            case ACCR_LOR: d.wcode = W_LOR; d.ident = 0; break;
            }
        } else {
            const bool wide = in_type == ACCR_F32 && acc == ACCR_F64;
            switch (op) {
            case ACCR_ADD:
                if (wide) { d.wcode = W_ADDF_WIDE; d.ident = d2u(-0.0); }
                else if (in_type == ACCR_F32 && (flags & ACCR_COMPENSATED)) { d.wcode = W_ADDF_COMP; d.ident = f2u(-0.0f); }
                else { d.wcode = W_ADDF; d.ident = e64 ? d2u(-0.0) : f2u(-0.0f); }
                break;
            case ACCR_MUL:
                if (wide) { d.wcode = W_MULF_WIDE; d.ident = d2u(1.0); }
                else { d.wcode = W_MULF; d.ident = e64 ? d2u(1.0) : f2u(1.0f); }
                break;
            case ACCR_MAX:
                d.wcode = W_MAXF;
                d.ident = e64 ? (uint64_t)fkey64(d2u(-INFINITY)) : (uint64_t)(uint32_t)fkey32(f2u(-INFINITY));
                break;
            case ACCR_MIN:
                d.wcode = W_MINF;
                d.ident = e64 ? (uint64_t)fkey64(d2u(INFINITY)) : (uint64_t)(uint32_t)fkey32(f2u(INFINITY));
                break;
            }
        }
        if (c[k].init) {
            if (a64) memcpy(&d.init, c[k].init, 8);
            else { uint32_t v; memcpy(&v, c[k].init, 4); d.init = v; }
        } else {
            d.init = var_identity(op, acc);
        }
    }
    return ACCR_OK;
}

}  // namespace accr
