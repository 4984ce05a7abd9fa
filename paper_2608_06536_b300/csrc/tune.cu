// Autotuner cache: the fastest measured configuration per shape bucket,
// shared by every handle in the process, with a text form for saving it
// between processes.  The timing itself lives with the entry points
// (jk_api.cu), which own problem validation and dispatch.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>

#include "jk_internal.h"

namespace jk {

namespace {

struct Entry {
    jk_tune_config cfg;
    double ms;
};

std::mutex g_mu;
std::map<TuneKey, Entry> g_cache;

int ceil_div(long long x, int q) { return static_cast<int>((x + q - 1) / q); }

bool valid_cfg(const jk_tune_config &c) {
    return c.aux_chunk >= 0 && (c.schedule == 0 || c.schedule == 1) && (c.raster == 0 || c.raster == 1) &&
           (c.tile == 0 || c.tile == 1);
}

}  // namespace

bool TuneKey::operator<(const TuneKey &o) const {
    return std::tie(op, prec, sms, nmol, nb, nauxb, nd, ksumb) <
           std::tie(o.op, o.prec, o.sms, o.nmol, o.nb, o.nauxb, o.nd, o.ksumb);
}

// Bucket: largest nbf in steps of 32, total naux in steps of 256, total
// density count, total width in steps of 16, molecule count, SM count.
TuneKey tune_key(jk_op op, jk_precision p, int sms, int nmol, const Problem *pbs) {
    TuneKey k{};
    k.op = static_cast<int>(op);
    k.prec = static_cast<int>(p);
    k.sms = sms;
    k.nmol = nmol;
    int nmax = 0, nd = 0;
    long long naux = 0, ksum = 0;
    for (int m = 0; m < nmol; m++) {
        nmax = std::max(nmax, pbs[m].n);
        nd += pbs[m].nd;
        naux += pbs[m].naux;
        ksum += pbs[m].ksum;
    }
    k.nb = ceil_div(nmax, 32);
    k.nauxb = ceil_div(naux, 256);
    k.nd = nd;
    k.ksumb = ceil_div(ksum, 16);
    return k;
}

bool tune_lookup(const TuneKey &k, jk_tune_config &cfg) {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = g_cache.find(k);
    if (it == g_cache.end()) return false;
    cfg = it->second.cfg;
    return true;
}

void tune_store(const TuneKey &k, const jk_tune_config &cfg, double ms) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache[k] = Entry{cfg, ms};
}

}  // namespace jk

using namespace jk;

extern "C" {

jk_status jk_tune_export(char *buf, size_t cap, size_t *len) {
    std::string out;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        char line[256];
        for (const auto &kv : g_cache) {
            const TuneKey &k = kv.first;
            const Entry &e = kv.second;
            std::snprintf(line, sizeof line, "jk-tune 4 %d %d %d %d %d %d %d %d %d %d %d %d %.6f\n", k.op,
                          k.prec, k.sms, k.nmol, k.nb, k.nauxb, k.nd, k.ksumb, e.cfg.aux_chunk, e.cfg.schedule,
                          e.cfg.raster, e.cfg.tile, e.ms);
            out += line;
        }
    }
    if (len) *len = out.size();
    if (buf && cap > 0) {
        const size_t n = std::min(cap - 1, out.size());
        std::memcpy(buf, out.data(), n);
        buf[n] = '\0';
    }
    return JK_OK;
}

jk_status jk_tune_import(const char *text) {
    if (!text) return JK_ERR_ARG;
    const char *p = text;
    while (*p) {
        const char *eol = std::strchr(p, '\n');
        const size_t n = eol ? static_cast<size_t>(eol - p) : std::strlen(p);
        std::string line(p, n);
        p += n + (eol ? 1 : 0);
        const size_t first = line.find_first_not_of(" \t\r");
        if (first == std::string::npos || line[first] == '#') continue;
        TuneKey k{};
        jk_tune_config c{};
        int ver = 0, used = 0;
        double ms = 0.0;
        const int got = std::sscanf(line.c_str(),  " jk-tune %d %d %d %d %d %d %d %d %d %d %d %d %d %lf %n", &ver,
                                    &k.op, &k.prec, &k.sms, &k.nmol, &k.nb, &k.nauxb, &k.nd, &k.ksumb,
                                    &c.aux_chunk, &c.schedule, &c.raster, &c.tile, &ms, &used);
        if (got != 14 || ver != 4 || static_cast<size_t>(used) != line.size() || !valid_cfg(c) ||
            !std::isfinite(ms))
            return JK_ERR_ARG;
        tune_store(k, c, ms);
    }
    return JK_OK;
}

jk_status jk_tune_clear(void) {
    std::lock_guard<std::mutex> lock(g_mu);
    g_cache.clear();
    return JK_OK;
}

}  // extern "C"
