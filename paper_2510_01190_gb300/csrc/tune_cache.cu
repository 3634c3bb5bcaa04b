// Autotuner cache: the tile shape lcp_batch_autotune picked for a batch of a
// given shape on a given device, kept in a small JSON file so that a later call
// (or another process) takes it without timing every shape again.
//
// The file is this library's own format, one object:
//   {"lcp_tune_cache": 1, "entries": [
//     {"key": "<device>|sm<n>|...", "tile": [rows, cols], "ms": [t0, t1, t2, t3]},
//     ...
//   ]}
// with `ms` the timed mean of each shape in the order of lcp_tune's list.  It is
// rewritten whole on every store: into `<path>.tmp.<pid>`, then renamed over the
// file, so that a reader never sees a half-written cache.  A missing, empty or
// malformed file reads as empty.  Host code only.
#include <unistd.h>

#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "lcp_common.cuh"

namespace lcp {
namespace {

constexpr int kNumShapes = 4;
constexpr int kShapeRows[kNumShapes] = {64, 32, 32, 16};
constexpr int kShapeCols[kNumShapes] = {64, 128, 64, 128};

struct Entry {
    std::string key;
    int rows = 0, cols = 0;
    float ms[kNumShapes] = {0.f, 0.f, 0.f, 0.f};
};

bool known_shape(int rows, int cols) {
    for (int s = 0; s < kNumShapes; ++s)
        if (kShapeRows[s] == rows && kShapeCols[s] == cols) return true;
    return false;
}

std::string escape(const std::string& s) {
    std::string o;
    for (const char ch : s) {
        const unsigned char c = static_cast<unsigned char>(ch);
        if (c == '"' || c == '\\') {
            o += '\\';
            o += ch;
        } else if (c < 0x20) {
            char buf[8];
            std::snprintf(buf, sizeof(buf), "\\u%04x", c);
            o += buf;
        } else {
            o += ch;
        }
    }
    return o;
}

bool read_file(const char* path, std::string& text) {
    FILE* f = std::fopen(path, "rb");
    if (!f) return false;
    char buf[4096];
    size_t n;
    while ((n = std::fread(buf, 1, sizeof(buf), f)) > 0) text.append(buf, n);
    std::fclose(f);
    return true;
}

// A JSON string starting at text[i] == '"' (the escapes this file writes); i ends
// past the closing quote.  False when the string is not closed.
bool parse_string(const std::string& text, size_t& i, std::string& out) {
    if (i >= text.size() || text[i] != '"') return false;
    out.clear();
    for (++i; i < text.size(); ++i) {
        const char c = text[i];
        if (c == '"') {
            ++i;
            return true;
        }
        if (c != '\\') {
            out += c;
            continue;
        }
        if (++i >= text.size()) return false;
        const char e = text[i];
        if (e == 'u') {
            if (i + 4 >= text.size()) return false;
            out += static_cast<char>(std::strtol(text.substr(i + 1, 4).c_str(), nullptr, 16));
            i += 4;
        } else {
            out += e;  // \" and \\ (the only other escapes written)
        }
    }
    return false;
}

// The numbers of a JSON array starting at the first '[' at or after i.
bool parse_numbers(const std::string& text, size_t& i, std::vector<double>& out) {
    i = text.find('[', i);
    if (i == std::string::npos) return false;
    out.clear();
    const size_t end = text.find(']', i);
    if (end == std::string::npos) return false;
    const char* p = text.c_str() + i + 1;
    const char* stop = text.c_str() + end;
    while (p < stop) {
        while (p < stop && (*p == ' ' || *p == ',' || *p == '\n' || *p == '\t' || *p == '\r')) ++p;
        if (p >= stop) break;
        char* q = nullptr;
        const double v = std::strtod(p, &q);
        if (q == p) return false;
        out.push_back(v);
        p = q;
    }
    i = end + 1;
    return true;
}

// Every well-formed entry of the file, in order; parsing stops at the first one
// that is not.
std::vector<Entry> parse(const std::string& text) {
    std::vector<Entry> out;
    size_t i = 0;
    for (;;) {
        i = text.find("\"key\"", i);
        if (i == std::string::npos) break;
        i = text.find('"', i + 5);
        Entry e;
        std::vector<double> nums;
        if (i == std::string::npos || !parse_string(text, i, e.key)) break;
        size_t t = text.find("\"tile\"", i);
        if (t == std::string::npos || !parse_numbers(text, t, nums) || nums.size() != 2) break;
        e.rows = static_cast<int>(nums[0]);
        e.cols = static_cast<int>(nums[1]);
        size_t m = text.find("\"ms\"", t);
        if (m == std::string::npos || !parse_numbers(text, m, nums) || nums.size() != kNumShapes) break;
        for (int s = 0; s < kNumShapes; ++s) e.ms[s] = static_cast<float>(nums[s]);
        out.push_back(e);
        i = m;
    }
    return out;
}

bool write_entries(const char* path, const std::vector<Entry>& entries) {
    const std::string tmp = std::string(path) + ".tmp." + std::to_string(static_cast<long>(getpid()));
    FILE* f = std::fopen(tmp.c_str(), "wb");
    if (!f) return false;
    bool ok = std::fprintf(f, "{\"lcp_tune_cache\": 1, \"entries\": [\n") > 0;
    for (size_t k = 0; k < entries.size() && ok; ++k) {
        const Entry& e = entries[k];
        ok = std::fprintf(f, "  {\"key\": \"%s\", \"tile\": [%d, %d], \"ms\": [%.6g, %.6g, %.6g, %.6g]}%s\n",
                          escape(e.key).c_str(), e.rows, e.cols, e.ms[0], e.ms[1], e.ms[2], e.ms[3],
                          k + 1 < entries.size() ? "," : "") > 0;
    }
    ok = ok && std::fprintf(f, "]}\n") > 0;
    ok = (std::fclose(f) == 0) && ok;
    if (!ok || std::rename(tmp.c_str(), path) != 0) {
        std::remove(tmp.c_str());
        return false;
    }
    return true;
}

const char* resolve_path(const char* path) {
    if (path && *path) return path;
    const char* env = std::getenv("LCP_TUNE_CACHE");
    return env && *env ? env : nullptr;
}

}  // namespace
}  // namespace lcp

using namespace lcp;

extern "C" int lcp_tune_cache_lookup(const char* path, const char* key, lcp_tune* best, float* ms) {
    if (!path || !*path || !key || !best) return fail(LCP_ERR_ARG, "lcp_tune_cache_lookup: NULL path, key or best");
    std::string text;
    if (!read_file(path, text)) return 0;
    const std::vector<Entry> entries = parse(text);
    for (size_t k = entries.size(); k-- > 0;) {  // the last record of a key wins
        const Entry& e = entries[k];
        if (e.key != key) continue;
        if (!known_shape(e.rows, e.cols)) return 0;
        best->tile_rows = e.rows;
        best->tile_cols = e.cols;
        best->ctas_per_sm = 0;
        if (ms)
            for (int s = 0; s < kNumShapes; ++s) ms[s] = e.ms[s];
        return 1;
    }
    return 0;
}

extern "C" lcp_status lcp_tune_cache_store(const char* path, const char* key, const lcp_tune* best, const float* ms) {
    if (!path || !*path || !key || !best) return fail(LCP_ERR_ARG, "lcp_tune_cache_store: NULL path, key or best");
    if (!known_shape(best->tile_rows, best->tile_cols))
        return fail(LCP_ERR_ARG, "lcp_tune_cache_store: tile %d x %d is not one of the batch kernel's shapes",
                    best->tile_rows, best->tile_cols);
    std::string text;
    std::vector<Entry> entries;
    if (read_file(path, text)) entries = parse(text);
    Entry e;
    e.key = key;
    e.rows = best->tile_rows;
    e.cols = best->tile_cols;
    if (ms)
        for (int s = 0; s < kNumShapes; ++s) e.ms[s] = ms[s];
    bool replaced = false;
    for (Entry& x : entries)
        if (x.key == e.key) {
            x = e;
            replaced = true;
        }
    if (!replaced) entries.push_back(e);
    if (!write_entries(path, entries))
        return fail(LCP_ERR_ARG, "lcp_tune_cache_store: cannot write %s: %s", path, std::strerror(errno));
    return LCP_OK;
}

extern "C" int lcp_batch_tune_key(const lcp_batch_plan* plan, char* buf, size_t len) {
    if (!plan || !buf || len == 0) return fail(LCP_ERR_ARG, "lcp_batch_tune_key: NULL plan or buffer");
    int dev = 0, sms = 0;
    cudaDeviceProp prop;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return fail(LCP_ERR_CUDA, "lcp_batch_tune_key: no device");
    }
    const int n = std::snprintf(buf, len, "%s|sm%d|in%d|out%d|fields%d|iso%d|cells%lld|ciso%lld|mbytes%lld", prop.name,
                                sms, static_cast<int>(plan->in_dtype), static_cast<int>(plan->out_dtype), plan->n_fields,
                                plan->n_iso, static_cast<long long>(plan->cells),
                                static_cast<long long>(plan->cell_isovalues), static_cast<long long>(plan->member_bytes));
    if (n < 0 || static_cast<size_t>(n) >= len) return fail(LCP_ERR_ARG, "lcp_batch_tune_key: buffer of %zu bytes too small", len);
    return n;
}

extern "C" lcp_status lcp_batch_autotune_cached(const lcp_batch_plan* plan, int reps, const char* cache_path,
                                                lcp_tune* best, float* ms, int* from_cache, lcp_stream_t stream) {
    if (!plan || !best) return fail(LCP_ERR_ARG, "lcp_batch_autotune_cached: NULL plan or best");
    if (from_cache) *from_cache = 0;
    const char* path = resolve_path(cache_path);
    char key[512];
    if (path) {
        const int n = lcp_batch_tune_key(plan, key, sizeof(key));
        if (n < 0) return static_cast<lcp_status>(n);
        const int hit = lcp_tune_cache_lookup(path, key, best, ms);
        if (hit < 0) return static_cast<lcp_status>(hit);
        if (hit == 1) {
            if (from_cache) *from_cache = 1;
            return LCP_OK;
        }
    }
    float t[kNumShapes];
    const lcp_status s = lcp_batch_autotune(plan, reps, best, t, stream);
    if (s != LCP_OK) return s;
    if (ms)
        for (int k = 0; k < kNumShapes; ++k) ms[k] = t[k];
    return path ? lcp_tune_cache_store(path, key, best, t) : LCP_OK;
}
