// Process-wide table of tuned launch parameters (usfft_autotune fills it; the launchers read it).
//
// Only parameters that leave every result bit-identical are tuned: the persistent grid size of the
// 2-D samplers (each system is solved by one CTA whatever the grid) and the column-pair tile of the
// two-pass lattice FFT (each column's transform is the same arithmetic whatever the tile).  Keys:
//   TUNE_SAMPLER_BLOCKS: precision * 64 + (n + 15) / 16  (transform-size bucket of the mesh)
//   TUNE_FFT_TILE:       2 * L + (final pass ? 1 : 0)     (sub-transform length and pass)
// Text form, one entry per line: "<knob> <key> <value> <ms>".
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "usfft_internal.h"

namespace usfft {

namespace {
struct Entry {
    int value;
    double ms;
};
std::mutex g_tune_mu;
std::map<std::pair<int, int64_t>, Entry> g_tune;
}  // namespace

int tune_get(int knob, int64_t key, int fallback) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune.find({knob, key});
    return it == g_tune.end() ? fallback : it->second.value;
}

void tune_set(int knob, int64_t key, int value, double ms) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune[{knob, key}] = Entry{value, ms};
}

void tune_erase(int knob, int64_t key) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.erase({knob, key});
}

std::string tune_dump() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    std::string out;
    char line[128];
    for (const auto& kv : g_tune) {
        snprintf(line, sizeof line, "%d %lld %d %.6f\n", kv.first.first, (long long)kv.first.second, kv.second.value,
                 kv.second.ms);
        out += line;
    }
    return out;
}

// every line must parse as four fields with a known knob and a positive value; nothing is stored
// unless the whole text parses
bool tune_parse(const char* text, std::string& err) {
    std::map<std::pair<int, int64_t>, Entry> add;
    const char* p = text;
    int lineno = 0;
    while (p && *p) {
        const char* nl = strchr(p, '\n');
        std::string ln(p, nl ? (size_t)(nl - p) : strlen(p));
        p = nl ? nl + 1 : nullptr;
        ++lineno;
        if (ln.find_first_not_of(" \t\r") == std::string::npos) continue;
        int knob = 0, value = 0;
        long long key = 0;
        double ms = 0.0;
        char extra = 0;
        if (sscanf(ln.c_str(), "%d %lld %d %lf %c", &knob, &key, &value, &ms, &extra) != 4 ||
            (knob != TUNE_SAMPLER_BLOCKS && knob != TUNE_FFT_TILE) || value < 1 || value > (1 << 20)) {
            err = "tune table line " + std::to_string(lineno) + ": expected '<knob> <key> <value> <ms>'";
            return false;
        }
        add[{knob, (int64_t)key}] = Entry{value, ms};
    }
    std::lock_guard<std::mutex> lk(g_tune_mu);
    for (const auto& kv : add) g_tune[kv.first] = kv.second;
    return true;
}

void tune_clear() {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune.clear();
}

}  // namespace usfft
