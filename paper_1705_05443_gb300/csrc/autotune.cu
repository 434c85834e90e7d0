// autotune.cu -- the table of measured launch choices.
//
// A launch site with several valid configurations (threads per node CTA of
// the compression, source tile and target block of the kernel sums) names
// its shape by a key.  With tuning on, the first launch of a key times every
// candidate on the launching stream and records the fastest; afterwards, and
// with tuning off, the recorded choice is used, else the site's default.
// The table is process-wide and can be saved to and loaded from a flat JSON
// file:  {"smash_autotune": 1, "entries": {"key": value, ...}}.  The file
// named by the environment variable SMASH_AUTOTUNE_CACHE is loaded at the
// first lookup.
#include <cctype>
#include <cstdlib>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>

#include "internal.cuh"

namespace smash {

namespace {
std::mutex g_mu;
std::map<std::string, int> g_table;
std::map<std::string, int> g_force;  // key prefix -> forced candidate
std::atomic<int> g_mode{0};
bool g_env_loaded = false;

// entries of the flat JSON format above; returns -1 on a malformed file
int parse_into(const std::string &text, std::map<std::string, int> &out) {
    size_t p = text.find("\"entries\"");
    if (p == std::string::npos) return -1;
    p = text.find('{', p);
    if (p == std::string::npos) return -1;
    int n = 0;
    ++p;
    for (;;) {
        while (p < text.size() && (std::isspace((unsigned char)text[p]) || text[p] == ',')) ++p;
        if (p >= text.size()) return -1;
        if (text[p] == '}') return n;
        if (text[p] != '"') return -1;
        size_t q = text.find('"', p + 1);
        if (q == std::string::npos) return -1;
        std::string key = text.substr(p + 1, q - p - 1);
        p = text.find(':', q);
        if (p == std::string::npos) return -1;
        ++p;
        while (p < text.size() && std::isspace((unsigned char)text[p])) ++p;
        size_t e = p;
        if (e < text.size() && text[e] == '-') ++e;
        while (e < text.size() && std::isdigit((unsigned char)text[e])) ++e;
        if (e == p) return -1;
        out[key] = std::atoi(text.substr(p, e - p).c_str());
        ++n;
        p = e;
    }
}

int load_file(const char *path) {
    std::ifstream f(path);
    if (!f) return -1;
    std::stringstream ss;
    ss << f.rdbuf();
    std::map<std::string, int> tmp;
    int n = parse_into(ss.str(), tmp);
    if (n < 0) return -1;
    for (auto &kv : tmp) g_table[kv.first] = kv.second;
    return n;
}

void load_env_locked() {
    if (g_env_loaded) return;
    g_env_loaded = true;
    const char *p = std::getenv("SMASH_AUTOTUNE_CACHE");
    if (p && *p) load_file(p);
}
}  // namespace

bool tune_active(cudaStream_t s) {
    if (!g_mode.load()) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return cs == cudaStreamCaptureStatusNone;
}

bool tune_find(const std::string &key, int &value) {
    std::lock_guard<std::mutex> lock(g_mu);
    load_env_locked();
    auto it = g_table.find(key);
    if (it == g_table.end()) return false;
    value = it->second;
    return true;
}

void tune_put(const std::string &key, int value) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_table[key] = value;
}

float tune_time(cudaStream_t s, const std::function<void()> &launch, int reps) {
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    launch();  // warm-up
    CK(cudaEventRecord(a, s));
    for (int i = 0; i < reps; ++i) launch();
    CK(cudaEventRecord(b, s));
    CK(cudaEventSynchronize(b));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b));
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms / (float)reps;
}

int tune_choose(const std::string &key, const std::vector<int> &cands, int dflt, cudaStream_t s,
                const std::function<void(int)> &launch) {
    int v = dflt;
    {
        int forced = -1;
        {
            std::lock_guard<std::mutex> lock(g_mu);
            for (auto &kv : g_force)
                if (key.compare(0, kv.first.size(), kv.first) == 0) forced = kv.second;
        }
        if (forced >= 0 && std::find(cands.begin(), cands.end(), forced) != cands.end()) {
            launch(forced);
            return forced;
        }
    }
    if (tune_find(key, v)) {
        if (std::find(cands.begin(), cands.end(), v) == cands.end()) v = dflt;  // stale entry
        launch(v);
        return v;
    }
    if (!tune_active(s) || cands.size() < 2) {
        launch(dflt);
        return dflt;
    }
    float best = 0.f;
    int bc = dflt;
    for (size_t i = 0; i < cands.size(); ++i) {
        const int c = cands[i];
        float ms = tune_time(s, [&] { launch(c); }, 2);
        if (i == 0 || ms < best) { best = ms; bc = c; }
    }
    tune_put(key, bc);
    launch(bc);  // the output of the chosen configuration
    return bc;
}

}  // namespace smash

extern "C" {

void smash_set_autotune(int on) { smash::g_mode.store(on ? 1 : 0); }

int smash_autotune_entries(void) {
    std::lock_guard<std::mutex> lock(smash::g_mu);
    smash::load_env_locked();
    return (int)smash::g_table.size();
}

void smash_autotune_clear(void) {
    std::lock_guard<std::mutex> lock(smash::g_mu);
    smash::g_env_loaded = true;
    smash::g_table.clear();
}

int smash_autotune_load(const char *path) {
    if (!path) {
        smash::set_last_error("path is NULL");
        return -1;
    }
    std::lock_guard<std::mutex> lock(smash::g_mu);
    smash::g_env_loaded = true;
    int n = smash::load_file(path);
    if (n < 0) smash::set_last_error("cannot read an autotune table from this file");
    return n;
}

smash_status smash_autotune_save(const char *path) {
    if (!path) {
        smash::set_last_error("path is NULL");
        return SMASH_EINVAL;
    }
    std::lock_guard<std::mutex> lock(smash::g_mu);
    std::ofstream f(path);
    if (!f) {
        smash::set_last_error("cannot open the file for writing");
        return SMASH_EINVAL;
    }
    f << "{\"smash_autotune\": 1, \"entries\": {";
    bool first = true;
    for (auto &kv : smash::g_table) {
        f << (first ? "\n  " : ",\n  ") << '"' << kv.first << "\": " << kv.second;
        first = false;
    }
    f << "\n}}\n";
    return f ? SMASH_OK : SMASH_EINVAL;
}

void smash_autotune_force(const char *prefix, int value) {
    if (!prefix) return;
    std::lock_guard<std::mutex> lock(smash::g_mu);
    if (value < 0) smash::g_force.erase(prefix);
    else smash::g_force[prefix] = value;
}

int smash_autotune_lookup(const char *key, int *value) {
    if (!key || !value) return 0;
    int v = 0;
    if (!smash::tune_find(key, v)) return 0;
    *value = v;
    return 1;
}

}  // extern "C"
