// Project-written autotuner: the counterpart of the guide's FFTW planning modes (digHoloConfigSetFFTWPlanMode)
// and wisdom file (digHoloFFTWWisdomFilename).  For one geometry it times each candidate way of computing the
// same reconstruction -- the kernel variant, the generic path's launch chunk size, the radix plan of the
// M-point inverse transforms -- with CUDA events on the caller's frames, keeps the fastest and files the choice
// under a geometry key in a JSON cache that later runs load instead of searching again.
#include <cuda_runtime.h>

#include <algorithm>
#include <cctype>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

#include "runtime.hpp"

namespace dh {

int process(Handle* H, const void* frames, int dtype, int batch, void* window, void* fields, void* coefs,
            cudaStream_t st);

namespace {

const int kRadices[] = {2, 3, 4, 5, 7, 8, 11, 13, 16, 17, 19};
const int kChunkMb[] = {24, 48, 96};

bool radix_ok(int r) { return std::find(std::begin(kRadices), std::end(kRadices), r) != std::end(kRadices); }

bool plan_ok(const std::vector<int>& plan, int m) {
    if (plan.empty() || (int)plan.size() > DH_MAX_RADICES) return false;
    long long prod = 1;
    for (int r : plan) {
        if (!radix_ok(r)) return false;
        prod *= r;
    }
    return prod == m;
}

std::vector<int> tuning_plan(const dh_tuning& t) { return std::vector<int>(t.radix, t.radix + t.nradix); }

dh_tuning make_tuning(int variant, int chunk_mb, const std::vector<int>& plan) {
    dh_tuning t;
    std::memset(&t, 0, sizeof t);
    t.variant = variant;
    t.chunk_mb = chunk_mb;
    t.nradix = (int)plan.size();
    for (int i = 0; i < t.nradix; ++i) t.radix[i] = plan[i];
    return t;
}

// Power-of-two factorisations into radices 2..16 tried besides the default one, per exponent.
std::vector<std::vector<int>> pow2_alternatives(int e) {
    switch (e) {
        case 4: return {{4, 4}};
        case 5: return {{4, 8}, {16, 2}};
        case 6: return {{16, 4}, {4, 16}};
        case 7: return {{8, 16}, {8, 4, 4}};
        case 8: return {{8, 8, 4}, {4, 8, 8}};
        case 9: return {{16, 16, 2}, {16, 8, 4}};
        case 10: return {{8, 8, 16}, {16, 16, 4}};
        default: return {};
    }
}

// The default radix plan of M and up to three alternatives (reversed; other power-of-two factorisations with
// the odd primes kept last), without duplicates.
std::vector<std::vector<int>> m_plans(int m) {
    std::vector<std::vector<int>> out;
    const std::vector<int> def = radix_plan(m);
    if (def.empty()) return out;
    out.push_back(def);
    auto add = [&](const std::vector<int>& p) {
        if (out.size() < 4 && plan_ok(p, m) && std::find(out.begin(), out.end(), p) == out.end()) out.push_back(p);
    };
    add(std::vector<int>(def.rbegin(), def.rend()));
    int odd = m, e = 0;
    while (odd % 2 == 0) { odd /= 2; ++e; }
    std::vector<int> primes;
    for (int r : def)
        if (r % 2) primes.push_back(r);
    for (const auto& p2 : pow2_alternatives(e)) {
        std::vector<int> p = p2;
        p.insert(p.end(), primes.begin(), primes.end());
        add(p);
    }
    return out;
}

// ---------------------------------------------------------------------------------------------- JSON cache
// {"format": "digholo-gb300-tuning", "version": 1, "entries": [{"key": "...", "variant": v, "chunk_mb": c,
//  "radix": [..], "ms": t, ...}, ...]}: a small reader for exactly this shape (objects, arrays, strings,
// numbers, true / false / null), and a writer.

struct JValue {
    enum Kind { NUL, NUM, STR, ARR, OBJ, BOOL } kind = NUL;
    double num = 0;
    std::string str;
    std::vector<JValue> arr;
    std::vector<std::pair<std::string, JValue>> obj;
    const JValue* get(const std::string& k) const {
        for (const auto& kv : obj)
            if (kv.first == k) return &kv.second;
        return nullptr;
    }
};

struct JParser {
    const std::string& s;
    size_t i = 0;
    explicit JParser(const std::string& src) : s(src) {}
    void ws() {
        while (i < s.size() && std::isspace((unsigned char)s[i])) ++i;
    }
    bool lit(const char* w) {
        const size_t n = std::strlen(w);
        if (s.compare(i, n, w) != 0) return false;
        i += n;
        return true;
    }
    bool string(std::string* out) {
        if (i >= s.size() || s[i] != '"') return false;
        ++i;
        out->clear();
        while (i < s.size() && s[i] != '"') {
            if (s[i] == '\\') {
                if (++i >= s.size()) return false;
                const char c = s[i];
                if (c == 'u') return false;   // keys and values here are plain ASCII
                out->push_back(c == 'n' ? '\n' : c == 't' ? '\t' : c);
            } else {
                out->push_back(s[i]);
            }
            ++i;
        }
        if (i >= s.size()) return false;
        ++i;
        return true;
    }
    bool value(JValue* v, int depth) {
        if (depth > 16) return false;
        ws();
        if (i >= s.size()) return false;
        const char c = s[i];
        if (c == '{') {
            v->kind = JValue::OBJ;
            ++i;
            ws();
            if (i < s.size() && s[i] == '}') { ++i; return true; }
            for (;;) {
                ws();
                std::string k;
                if (!string(&k)) return false;
                ws();
                if (i >= s.size() || s[i] != ':') return false;
                ++i;
                JValue e;
                if (!value(&e, depth + 1)) return false;
                v->obj.emplace_back(k, e);
                ws();
                if (i < s.size() && s[i] == ',') { ++i; continue; }
                if (i < s.size() && s[i] == '}') { ++i; return true; }
                return false;
            }
        }
        if (c == '[') {
            v->kind = JValue::ARR;
            ++i;
            ws();
            if (i < s.size() && s[i] == ']') { ++i; return true; }
            for (;;) {
                JValue e;
                if (!value(&e, depth + 1)) return false;
                v->arr.push_back(e);
                ws();
                if (i < s.size() && s[i] == ',') { ++i; continue; }
                if (i < s.size() && s[i] == ']') { ++i; return true; }
                return false;
            }
        }
        if (c == '"') {
            v->kind = JValue::STR;
            return string(&v->str);
        }
        if (lit("true")) { v->kind = JValue::BOOL; v->num = 1; return true; }
        if (lit("false")) { v->kind = JValue::BOOL; v->num = 0; return true; }
        if (lit("null")) { v->kind = JValue::NUL; return true; }
        const char* b = s.c_str() + i;
        char* e = nullptr;
        const double d = std::strtod(b, &e);
        if (e == b) return false;
        i += (size_t)(e - b);
        v->kind = JValue::NUM;
        v->num = d;
        return true;
    }
};

bool int_field(const JValue& o, const char* k, int* out) {
    const JValue* v = o.get(k);
    if (!v || v->kind != JValue::NUM || v->num != (double)(int)v->num) return false;
    *out = (int)v->num;
    return true;
}

// Parse a cache file's text into entries; false (and *why) for anything that is not the expected shape.
bool parse_cache(const std::string& text, std::map<std::string, dh_tuning>* out, std::string* why) {
    JValue root;
    JParser p(text);
    if (!p.value(&root, 0)) { *why = "tuning cache is not valid JSON"; return false; }
    p.ws();
    if (p.i != text.size()) { *why = "tuning cache has trailing content"; return false; }
    const JValue* fmt = root.kind == JValue::OBJ ? root.get("format") : nullptr;
    if (!fmt || fmt->kind != JValue::STR || fmt->str != "digholo-gb300-tuning") {
        *why = "tuning cache lacks \"format\": \"digholo-gb300-tuning\"";
        return false;
    }
    const JValue* ents = root.get("entries");
    if (!ents || ents->kind != JValue::ARR) { *why = "tuning cache lacks an \"entries\" array"; return false; }
    std::map<std::string, dh_tuning> m;
    for (const JValue& e : ents->arr) {
        const JValue* key = e.kind == JValue::OBJ ? e.get("key") : nullptr;
        int variant = 0, chunk = 0;
        if (!key || key->kind != JValue::STR || !int_field(e, "variant", &variant) || !int_field(e, "chunk_mb", &chunk)) {
            *why = "tuning cache entry needs \"key\", \"variant\" and \"chunk_mb\"";
            return false;
        }
        if (variant < DH_VARIANT_AUTO || variant > DH_VARIANT_FUSED_GROUPS || chunk < 0 || chunk > 4096) {
            *why = "tuning cache entry out of range";
            return false;
        }
        std::vector<int> plan;
        const JValue* rad = e.get("radix");
        if (rad) {
            if (rad->kind != JValue::ARR || rad->arr.size() > DH_MAX_RADICES) { *why = "tuning cache radix must be a short array"; return false; }
            for (const JValue& r : rad->arr) {
                if (r.kind != JValue::NUM || !radix_ok((int)r.num) || r.num != (double)(int)r.num) {
                    *why = "tuning cache radix holds an unsupported value";
                    return false;
                }
                plan.push_back((int)r.num);
            }
        }
        m[key->str] = make_tuning(variant, chunk, plan);
    }
    out->swap(m);
    return true;
}

std::string json_escape(const std::string& v) {
    std::string o;
    for (char c : v) {
        if (c == '"' || c == '\\') o.push_back('\\');
        o.push_back(c);
    }
    return o;
}

bool write_cache(const std::string& path, const std::map<std::string, dh_tuning>& m, const std::string& key,
                 double best_ms, int candidates) {
    std::ostringstream o;
    o << "{\n  \"format\": \"digholo-gb300-tuning\",\n  \"version\": 1,\n  \"entries\": [";
    bool first = true;
    for (const auto& kv : m) {
        const dh_tuning& t = kv.second;
        o << (first ? "\n" : ",\n") << "    {\"key\": \"" << json_escape(kv.first) << "\", \"variant\": " << t.variant
          << ", \"chunk_mb\": " << t.chunk_mb << ", \"radix\": [";
        for (int i = 0; i < t.nradix; ++i) o << (i ? ", " : "") << t.radix[i];
        o << "]";
        if (kv.first == key) o << ", \"ms\": " << best_ms << ", \"candidates\": " << candidates;
        o << "}";
        first = false;
    }
    o << "\n  ]\n}\n";
    const std::string tmp = path + ".tmp";
    {
        std::ofstream f(tmp, std::ios::binary | std::ios::trunc);
        if (!f) return false;
        f << o.str();
        if (!f) return false;
    }
    return std::rename(tmp.c_str(), path.c_str()) == 0;
}

}  // namespace
}  // namespace dh

namespace dh {

std::string tuning_key(const Settings& s, const Geometry& g) {
    char b[192];
    if (g.square())
        std::snprintf(b, sizeof b, "N%d_M%d_G%d_P%d_W%d_H%d_prec%d_basis%d", g.n, g.m, g.groups, g.pols, s.width, s.height,
                      s.precision, g.basis);
    else   // non-square windows or fields name both axes
        std::snprintf(b, sizeof b, "N%dx%d_M%dx%d_G%d_P%d_W%d_H%d_prec%d_basis%d", g.n, g.ny, g.m, g.my, g.groups, g.pols,
                      s.width, s.height, s.precision, g.basis);
    return b;
}

namespace {

void apply_tuning(Handle* H, const dh_tuning& t, int m) {
    H->tuned = t.variant;
    H->chunk_mb = t.chunk_mb;
    std::vector<int> plan = tuning_plan(t);
    if (!plan_ok(plan, m)) plan.clear();
    if (plan != H->s.radix_m) {
        H->s.radix_m = plan;
        H->dirty = true;
    }
}

// The tuning in effect for geometry g: the one set for its key, else the cache's entry, else zeros.
dh_tuning effective(const Handle* H, const std::string& key) {
    if (H->tune_set && H->tune_key == key) return make_tuning(H->tuned, H->chunk_mb, H->s.radix_m);
    auto it = H->tune_cache.find(key);
    return it != H->tune_cache.end() ? it->second : make_tuning(0, 0, {});
}

// Whether the pruned fused kernel has its table block for every polarisation of these settings.
bool pruned_applies(const Settings& s, const Geometry& g) {
    if (g.n != 128 || g.m != 64 || g.groups > 16 || s.precision != DH_PRECISION_FP32) return false;
    Tables t;
    build_tables(s, g, &t);
    for (int p = 0; p < g.pols; ++p)
        if (t.pol[p].pr.empty()) return false;
    return true;
}

std::vector<dh_tuning> candidates(const Settings& s, const Geometry& g) {
    std::vector<dh_tuning> out;
    const bool fused = g.n == 128 && g.square() && g.groups <= 16 &&
                       (s.precision == DH_PRECISION_FP32 ? (g.m == 32 || g.m == 48 || g.m == 64) : g.m == 64);
    if (fused) {
        if (g.m == 64 && s.precision == DH_PRECISION_FP32) out.push_back(make_tuning(DH_VARIANT_FUSED_GROUPS, 0, {}));
        out.push_back(make_tuning(DH_VARIANT_FUSED, 0, {}));
        if (pruned_applies(s, g)) out.push_back(make_tuning(DH_VARIANT_FUSED_PRUNED, 0, {}));
        out.push_back(make_tuning(DH_VARIANT_GENERIC, 0, {}));
        return out;
    }
    // 256 x 256 windows with 96 x 96 fields: the fused kernel (uint16 frames; other frames run the generic path
    // whatever the choice), then the generic path's chunk sizes and radix plans
    if (g.n == 256 && g.square() && g.m == 96 && g.groups <= 16 && g.pols <= 2)
        out.push_back(make_tuning(DH_VARIANT_FUSED, 0, {}));
    // non-square geometries: the chunk size only (their radix plans stay the defaults)
    for (int mb : kChunkMb)
        for (const auto& plan : g.square() ? m_plans(g.m) : std::vector<std::vector<int>>{radix_plan(g.m)})
            out.push_back(make_tuning(DH_VARIANT_GENERIC, mb, plan));
    return out;
}

int set_tuning(Handle* H, const dh_tuning* t, const Geometry& g, const std::string& key) {
    if (!t) {
        H->tune_set = false;
        H->tune_key.clear();
        apply_tuning(H, effective(H, key), g.m);
        H->tune_key = key;
        return DH_SUCCESS;
    }
    if (t->variant < DH_VARIANT_AUTO || t->variant > DH_VARIANT_FUSED_GROUPS)
        return fail(DH_ERROR_INVALIDARGUMENT, "tuning variant must be one of DH_VARIANT_*");
    if (t->chunk_mb < 0 || t->chunk_mb > 4096) return fail(DH_ERROR_INVALIDARGUMENT, "tuning chunk_mb must be in [0, 4096]");
    if (t->nradix < 0 || t->nradix > DH_MAX_RADICES)
        return fail(DH_ERROR_INVALIDARGUMENT, "tuning nradix must be in [0, DH_MAX_RADICES]");
    if (t->nradix > 0 && !plan_ok(tuning_plan(*t), g.m))
        return fail(DH_ERROR_INVALIDARGUMENT, "tuning radix plan: supported radices whose product is the field size M");
    apply_tuning(H, *t, g.m);
    H->tune_set = true;
    H->tune_key = key;
    return DH_SUCCESS;
}

}  // namespace

void tune_refresh(Handle* H, const Geometry& g) {
    const std::string key = tuning_key(H->s, g);
    if (H->tune_set && H->tune_key == key) return;
    H->tune_set = false;
    H->tune_key = key;
    apply_tuning(H, effective(H, key), g.m);
}

}  // namespace dh

using namespace dh;

#define GET_HANDLE(h)                                                     \
    Handle* H = get_handle(h);                                            \
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "invalid handle");      \
    std::lock_guard<std::mutex> lk(H->mu)

extern "C" {

int dh_tuning_key(dh_handle h, char* buf, int len) {
    GET_HANDLE(h);
    if (!buf) return fail(DH_ERROR_NULLPOINTER, "buf is null");
    Geometry g;
    std::string why;
    int rc = build_geometry(H->s, &g, &why);
    if (rc) return fail(rc, why);
    const std::string key = tuning_key(H->s, g);
    if (len < (int)key.size() + 1) return fail(DH_ERROR_INVALIDARGUMENT, "buf too short for the tuning key");
    std::memcpy(buf, key.c_str(), key.size() + 1);
    return DH_SUCCESS;
}

int dh_tuning_candidates(dh_handle h, dh_tuning* out, int max, int* count) {
    GET_HANDLE(h);
    if (!count || (!out && max > 0)) return fail(DH_ERROR_NULLPOINTER, "count or out is null");
    Geometry g;
    std::string why;
    int rc = build_geometry(H->s, &g, &why);
    if (rc) return fail(rc, why);
    Settings s = H->s;
    s.radix_m.clear();
    const std::vector<dh_tuning> c = candidates(s, g);
    for (int i = 0; i < (int)c.size() && i < max; ++i) out[i] = c[i];
    *count = (int)c.size();
    return DH_SUCCESS;
}

int dh_set_tuning(dh_handle h, const dh_tuning* t) {
    GET_HANDLE(h);
    Geometry g;
    std::string why;
    int rc = build_geometry(H->s, &g, &why);
    if (rc) return fail(rc, why);
    return set_tuning(H, t, g, tuning_key(H->s, g));
}

int dh_get_tuning(dh_handle h, dh_tuning* out) {
    GET_HANDLE(h);
    if (!out) return fail(DH_ERROR_NULLPOINTER, "out is null");
    Geometry g;
    std::string why;
    int rc = build_geometry(H->s, &g, &why);
    if (rc) return fail(rc, why);
    *out = effective(H, tuning_key(H->s, g));
    return DH_SUCCESS;
}

int dh_set_tuning_cache(dh_handle h, const char* path) {
    GET_HANDLE(h);
    if (!path) {
        H->tune_path.clear();
        H->tune_cache.clear();
        H->dirty = true;
        return DH_SUCCESS;
    }
    std::map<std::string, dh_tuning> m;
    std::ifstream f(path, std::ios::binary);
    if (f) {
        std::stringstream ss;
        ss << f.rdbuf();
        std::string why;
        if (!parse_cache(ss.str(), &m, &why)) return fail(DH_ERROR_INVALIDARGUMENT, why + " (" + path + ")");
    }
    H->tune_path = path;
    H->tune_cache.swap(m);
    H->dirty = true;   // the next call looks its geometry up in the loaded choices
    return DH_SUCCESS;
}

int dh_autotune(dh_handle h, const void* d_frames, int dtype, int batch, void* d_fields, void* d_coefs, void* stream,
                int reps) {
    GET_HANDLE(h);
    if (!d_frames) return fail(DH_ERROR_NULLPOINTER, "frames pointer is null");
    if (reps < 1) reps = 3;
    if (batch < 1) batch = 1;
    Geometry g;
    std::string why;
    int rc = build_geometry(H->s, &g, &why);
    if (rc) return fail(rc, why);
    const std::string key = tuning_key(H->s, g);
    Settings s0 = H->s;
    s0.radix_m.clear();
    const std::vector<dh_tuning> cand = candidates(s0, g);
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return fail(DH_ERROR_CUDA, "tuner events");
    }
    const int held = H->variant;   // a variant the caller holds the handle to does not restrict the search
    H->variant = DH_VARIANT_AUTO;
    int best = -1;
    float best_ms = 0.f;
    for (int i = 0; i < (int)cand.size() && rc == DH_SUCCESS; ++i) {
        rc = set_tuning(H, &cand[i], g, key);
        if (rc == DH_SUCCESS) rc = process(H, d_frames, dtype, batch, nullptr, d_fields, d_coefs, st);
        if (rc) break;
        cudaEventRecord(e0, st);
        for (int r = 0; r < reps && rc == DH_SUCCESS; ++r)
            rc = process(H, d_frames, dtype, batch, nullptr, d_fields, d_coefs, st);
        cudaEventRecord(e1, st);
        cudaError_t e = cudaEventSynchronize(e1);
        float ms = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess && rc == DH_SUCCESS) rc = cuda_fail(e, "tuner timing");
        ms /= (float)reps;
        if (rc == DH_SUCCESS && (best < 0 || ms < best_ms)) {
            best = i;
            best_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc == DH_SUCCESS && best >= 0) {
        rc = set_tuning(H, &cand[best], g, key);
        H->tune_cache[key] = cand[best];
        if (rc == DH_SUCCESS && !H->tune_path.empty() &&
            !write_cache(H->tune_path, H->tune_cache, key, best_ms, (int)cand.size()))
            rc = fail(DH_ERROR_ERROR, "could not write the tuning cache " + H->tune_path);
        if (rc == DH_SUCCESS) rc = process(H, d_frames, dtype, batch, nullptr, d_fields, d_coefs, st);
    }
    H->variant = held;
    return rc;
}

}  // extern "C"
