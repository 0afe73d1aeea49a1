// rs_tune.cpp -- the autotuner's table: launch-shape choices measured on the device and kept
// per shape bucket, in memory for the process and optionally in a JSON file.
//
// Keys name a kernel, the storage size of the factor's scalars, the number of boxes of the
// launch and the quarter-octave bucket of its largest box dimensions; values are the chosen
// settings (a CTA-group scale, a variant flag).  rs_autotune (rs_factor.cpp) fills it by timing
// whole factorizations under each candidate setting and keeping, level by level, the fastest.
#include <math.h>
#include <stdio.h>

#include <cmath>
#include <fstream>
#include <map>
#include <mutex>
#include <sstream>
#include <string>

#include "rs_host.h"

namespace rs {

namespace {
std::mutex g_tune_mutex;
std::map<std::string, double> g_tune;
}  // namespace

thread_local TuneTrial g_trial;

static int qbucket(int64_t v) { return v <= 0 ? 0 : (int)std::lround(4.0 * std::log2((double)v)); }

std::string tune_key(const char* what, int esz, int nb, int64_t m, int64_t r)
{
    std::ostringstream o;
    o << what << ".s" << esz << ".b" << nb << ".m" << qbucket(m) << ".r" << qbucket(r);
    return o.str();
}

double tune_get(const std::string& key, double dflt)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = g_tune.find(key);
    return it == g_tune.end() ? dflt : it->second;
}

void tune_set(const std::string& key, double v)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune[key] = v;
}

int tune_count()
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    return (int)g_tune.size();
}

}  // namespace rs

using namespace rs;

extern "C" {

int rs_tune_clear(void)
{
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune.clear();
    return RS_OK;
}

int rs_tune_count(void) { return tune_count(); }

// {"rs_tune": 1, "entries": {"key": value, ...}}
int rs_tune_save(const char* path)
{
    if (!path) return fail(RS_E_INVALID, "NULL path");
    std::map<std::string, double> copy;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        copy = g_tune;
    }
    std::ofstream f(path);
    if (!f) return fail(RS_E_INVALID, std::string("cannot write ") + path);
    f << "{\"rs_tune\": 1, \"entries\": {";
    bool first = true;
    char buf[64];
    for (const auto& kv : copy) {
        snprintf(buf, sizeof buf, "%.17g", kv.second);
        f << (first ? "" : ", ") << "\n  \"" << kv.first << "\": " << buf;
        first = false;
    }
    f << "\n}}\n";
    return f ? RS_OK : fail(RS_E_INVALID, std::string("write failed: ") + path);
}

// Reads the format rs_tune_save writes: every "key": number pair inside "entries" is merged
// into the table; anything else is an error that leaves the table unchanged.
int rs_tune_load(const char* path)
{
    if (!path) return fail(RS_E_INVALID, "NULL path");
    std::ifstream f(path);
    if (!f) return fail(RS_E_INVALID, std::string("cannot read ") + path);
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string s = ss.str();
    const size_t e = s.find("\"entries\"");
    if (s.find("\"rs_tune\"") == std::string::npos || e == std::string::npos)
        return fail(RS_E_INVALID, "not an rs_tune file");
    size_t p = s.find('{', e);
    if (p == std::string::npos) return fail(RS_E_INVALID, "malformed rs_tune file");
    std::map<std::string, double> got;
    ++p;
    while (true) {
        while (p < s.size() && (isspace((unsigned char)s[p]) || s[p] == ',')) ++p;
        if (p >= s.size()) return fail(RS_E_INVALID, "malformed rs_tune file");
        if (s[p] == '}') break;
        if (s[p] != '"') return fail(RS_E_INVALID, "malformed rs_tune file");
        const size_t q = s.find('"', p + 1);
        if (q == std::string::npos) return fail(RS_E_INVALID, "malformed rs_tune file");
        const std::string key = s.substr(p + 1, q - p - 1);
        p = s.find(':', q);
        if (p == std::string::npos) return fail(RS_E_INVALID, "malformed rs_tune file");
        ++p;
        char* end = nullptr;
        const double v = strtod(s.c_str() + p, &end);
        if (end == s.c_str() + p || !std::isfinite(v)) return fail(RS_E_INVALID, "malformed value in rs_tune file");
        p = (size_t)(end - s.c_str());
        got[key] = v;
    }
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    for (const auto& kv : got) g_tune[kv.first] = kv.second;
    return RS_OK;
}

}  // extern "C"
