// tune.cu -- the library's autotuner.
//
// Some launch parameters change only how the work is spread over the GPU,
// never a result: the number of row warps per TMEM lane quarter of the
// tcgen05 matvec (each kernel value and each column sum is formed the same
// way), the CTAs per SM of the persistent grouped kernels (each tile is
// computed the same way by whichever CTA takes it) and the threads per CTA
// of the FSAI build (each Gram entry and each step of the local Cholesky is
// the same sum in the same order).  For these the library picks the fastest
// candidate by timing: the first call with a given shape runs every
// candidate on its own operands (each run overwrites the same outputs with
// the same values), keeps the fastest, and records the choice under a key of
// (kernel, shape bucket, device: compute capability and SM count).  Kernels
// whose launches are captured into a graph (the grouped solves) are timed
// candidate by candidate before the capture; the others are tuned on their
// real calls (tune_run): the first call with a key runs the default, the next
// ones each candidate once, timed, and then the fastest is recorded, so no
// work is repeated for tuning.  Later calls launch the recorded choice.  The cache is
// process-wide and can be persisted to a text file (afn_tune_set_cache):
// one "key choice" line per entry.  Because every candidate gives the same
// bits, a result never depends on what the tuner picked.
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>
#include <vector>

#include "afn_internal.cuh"

namespace afn {

namespace {
struct TuneCache {
    std::mutex mu;
    std::map<std::string, int> m;
    std::string path;        // "" = not persisted
    // keys being tuned online (tune_run): calls seen, best time per candidate
    struct Trial {
        int calls = 0;
        std::vector<float> ms;
    };
    std::map<std::string, Trial> trials;
};

TuneCache &cache()
{
    static TuneCache c;
    return c;
}

bool valid_key(const std::string &k)
{
    if (k.empty() || k.size() > 200) return false;
    for (char ch : k)
        if (ch <= ' ' || ch > '~') return false;
    return true;
}

// caller holds the lock
bool save_locked(const TuneCache &c, const std::string &path)
{
    const std::string tmp = path + ".tmp";
    {
        std::ofstream f(tmp, std::ios::trunc);
        if (!f) return false;
        f << "# afn autotuner cache v1: key choice\n";
        for (const auto &kv : c.m) f << kv.first << ' ' << kv.second << '\n';
        if (!f) return false;
    }
    return std::rename(tmp.c_str(), path.c_str()) == 0;
}

// caller holds the lock; entries of the file are added to (and override) the map
bool load_locked(TuneCache &c, const std::string &path, int *count)
{
    std::ifstream f(path);
    if (!f) return false;
    std::string line;
    int n = 0;
    while (std::getline(f, line)) {
        if (line.empty() || line[0] == '#') continue;
        std::istringstream ls(line);
        std::string key;
        long v = 0;
        if (!(ls >> key >> v) || !valid_key(key) || v < 0 || v > 1000000) return false;
        c.m[key] = (int)v;
        ++n;
    }
    if (count) *count = n;
    return true;
}
}  // namespace

std::string tune_device_tag()
{
    int dev = 0, major = 0, minor = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
    cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    char b[48];
    snprintf(b, sizeof(b), "sm%d%dx%d", major, minor, sms);
    return b;
}

bool tune_lookup(const std::string &key, int *choice)
{
    TuneCache &c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    auto it = c.m.find(key);
    if (it == c.m.end()) return false;
    *choice = it->second;
    return true;
}

void tune_store(const std::string &key, int choice)
{
    TuneCache &c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    c.m[key] = choice;
    if (!c.path.empty()) save_locked(c, c.path);
}

int tune_pick(const std::string &key, int ncand, const std::function<void(int)> &run,
              cudaStream_t s, int fallback)
{
    // a recorded choice outside the candidates (a hand-edited cache file, a
    // key reused with fewer candidates) is ignored and the key tuned again
    int choice = fallback;
    if (tune_lookup(key, &choice) && choice >= 0 && choice < ncand) return choice;
    // no timing inside a stream capture: the default, without recording it
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return fallback;
    }
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return fallback;
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        return fallback;
    }
    // each candidate: one warm-up run, then the best of three timed runs; the
    // default is kept unless another candidate is faster by more than 2 %
    std::vector<float> best((size_t)ncand, -1.f);
    for (int c = 0; c < ncand; ++c) {
        run(c);                       // warm-up (first-launch costs)
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(a, s);
            run(c);
            cudaEventRecord(b, s);
            float ms = 0.f;
            if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            if (best[c] < 0.f || ms < best[c]) best[c] = ms;
        }
    }
    int bi = fallback;
    for (int c = 0; c < ncand; ++c) {
        if (best[c] < 0.f) continue;
        const float ref = (bi >= 0 && bi < ncand && best[bi] >= 0.f) ? best[bi] : -1.f;
        if (ref < 0.f || best[c] < 0.98f * ref) bi = c;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    tune_store(key, bi);
    return bi;
}

void tune_run(const std::string &key, int ncand, const std::function<void(int)> &run,
              cudaStream_t s, int fallback)
{
    int choice = fallback;
    if (tune_lookup(key, &choice) && choice >= 0 && choice < ncand) {
        run(choice);
        return;
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        run(fallback);
        return;
    }
    // the call's candidate: the default on the first call (its first-launch costs stay
    // out of the comparison), then each candidate once, timed
    TuneCache &c = cache();
    int cand;
    {
        std::lock_guard<std::mutex> lk(c.mu);
        auto f = c.m.find(key);          // decided by another thread meanwhile
        if (f != c.m.end() && f->second >= 0 && f->second < ncand) {
            cand = -2;
            choice = f->second;
        } else {
            TuneCache::Trial &t = c.trials[key];
            if (t.ms.empty()) t.ms.assign((size_t)ncand, -1.f);
            const int call = t.calls++;
            cand = call == 0 ? -1 : (call - 1) % ncand;
        }
    }
    if (cand == -2) {
        run(choice);
        return;
    }
    if (cand < 0) {
        run(fallback);
        return;
    }
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) {
        run(cand);
        return;
    }
    if (cudaEventCreate(&b) != cudaSuccess) {
        cudaEventDestroy(a);
        run(cand);
        return;
    }
    cudaEventRecord(a, s);
    run(cand);
    cudaEventRecord(b, s);
    float ms = -1.f;
    if (cudaEventSynchronize(b) != cudaSuccess || cudaEventElapsedTime(&ms, a, b) != cudaSuccess) {
        cudaGetLastError();
        ms = -1.f;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    bool decide = false;
    int bi = fallback;
    {
        std::lock_guard<std::mutex> lk(c.mu);
        // another thread with the same key may have decided (and dropped the
        // trial) while this call ran: then there is nothing left to record
        auto it = c.trials.find(key);
        if (it == c.trials.end() || it->second.ms.size() != (size_t)ncand) return;
        TuneCache::Trial &t = it->second;
        if (ms >= 0.f && (t.ms[cand] < 0.f || ms < t.ms[cand])) t.ms[cand] = ms;
        bool all = true;
        for (float v : t.ms) all = all && v >= 0.f;
        if (all || t.calls > 4 * ncand + 1) {
            for (int q = 0; q < ncand; ++q) {
                if (t.ms[q] < 0.f) continue;
                const float ref = (bi >= 0 && bi < ncand && t.ms[bi] >= 0.f) ? t.ms[bi] : -1.f;
                if (ref < 0.f || t.ms[q] < 0.98f * ref) bi = q;
            }
            c.trials.erase(key);
            decide = true;
        }
    }
    if (decide) tune_store(key, bi);
}

int log2_bucket(int64_t v)
{
    int b = 0;
    while (v > 1 && b < 62) {
        v >>= 1;
        ++b;
    }
    return b;
}

}  // namespace afn

using namespace afn;

extern "C" afn_status afn_tune_set_cache(const char *path)
{
    TuneCache &c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (!path || !path[0]) {
        c.path.clear();
        return AFN_OK;
    }
    std::ifstream probe(path);
    if (probe.good()) {
        probe.close();
        if (!load_locked(c, path, nullptr)) {
            set_error("afn_tune_set_cache: %s is not an autotuner cache", path);
            return AFN_ERR_ARG;
        }
    }
    c.path = path;
    if (!save_locked(c, c.path)) {
        set_error("afn_tune_set_cache: cannot write %s", path);
        c.path.clear();
        return AFN_ERR_ARG;
    }
    return AFN_OK;
}

extern "C" afn_status afn_tune_get(const char *key, int32_t *choice)
{
    if (!key || !choice) {
        set_error("afn_tune_get: NULL argument");
        return AFN_ERR_ARG;
    }
    int v = 0;
    if (!tune_lookup(key, &v)) {
        set_error("afn_tune_get: no entry for %s", key);
        return AFN_ERR_ARG;
    }
    *choice = v;
    return AFN_OK;
}

extern "C" afn_status afn_tune_put(const char *key, int32_t choice)
{
    if (!key || !valid_key(key) || choice < 0) {
        set_error("afn_tune_put: invalid key or choice");
        return AFN_ERR_ARG;
    }
    tune_store(key, choice);
    return AFN_OK;
}

extern "C" int32_t afn_tune_count(void)
{
    TuneCache &c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    return (int32_t)c.m.size();
}

extern "C" void afn_tune_clear(void)
{
    TuneCache &c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    c.m.clear();
    if (!c.path.empty()) save_locked(c, c.path);
}

extern "C" int32_t afn_tune_key(int32_t index, char *buf, int32_t len)
{
    TuneCache &c = cache();
    std::lock_guard<std::mutex> lk(c.mu);
    if (index < 0 || index >= (int32_t)c.m.size()) return -1;
    auto it = c.m.begin();
    std::advance(it, index);
    if (buf && len > 0) {
        snprintf(buf, (size_t)len, "%s", it->first.c_str());
    }
    return it->second;
}
