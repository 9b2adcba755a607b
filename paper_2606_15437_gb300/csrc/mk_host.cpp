// mk_host.cpp -- host helpers of the C ABI: error text, status decoding and
// census witness decoding.
#include <cstring>

#include "mk.h"

extern "C" const char *mk_strerror(int code) {
    switch (code) {
    case MK_OK: return "ok";
    case MK_E_SYNTAX: return "formula text does not parse";
    case MK_E_TOO_LONG: return "formula exceeds the node or instruction limit";
    case MK_E_VARS: return "variable index beyond p3";
    case MK_E_SLOTS: return "formula needs more registers than the program format holds";
    case MK_E_ARG: return "invalid argument or configuration";
    case MK_E_WORKSPACE: return "workspace missing or too small";
    case MK_E_CUDA: return "CUDA runtime error";
    case MK_E_PROGRAM: return "device found a malformed program";
    case MK_E_LIMIT: return "size limit exceeded (exhaustive valuations with k*n too large)";
    case MK_E_INTERNAL: return "internal consistency check failed";
    case MK_E_TIMEOUT: return "a bounded device wait ran out";
    default: return "unknown error";
    }
}

extern "C" int mk_status_error(int32_t status) {
    if (status == 0) return MK_OK;
    if (status & MK_ST_TIMEOUT) return MK_E_TIMEOUT;
    if (status & MK_ST_INTERNAL) return MK_E_INTERNAL;
    if (status & MK_ST_PROGRAM) return MK_E_PROGRAM;
    if (status & MK_ST_LIMIT) return MK_E_LIMIT;
    if (status & MK_ST_INDEX) return MK_E_ARG;
    return MK_E_INTERNAL;
}

extern "C" int mk_version(void) { return 1; }

extern "C" int mk_witness_cert(const mk_program *h_prog, const char *phi, uint32_t cls, int32_t n,
                               uint32_t samples, const uint32_t *h_samples_n, uint64_t key,
                               mk_cert *out) {
    if (!h_prog || !phi || !out || key == ~0ull) return MK_E_ARG;
    if (n < 1 || n > MK_MAX_WORLDS_EXH) return MK_E_ARG;
    int ci;
    switch (cls) {
    case MK_CLASS_K: ci = 0; break;
    case MK_CLASS_T: ci = 1; break;
    case MK_CLASS_S4: ci = 2; break;
    case MK_CLASS_S5: ci = 3; break;
    case MK_CLASS_K4: ci = 4; break;
    default: return MK_E_ARG;
    }
    const uint64_t f = key >> 27;
    const uint32_t j = (uint32_t)((key >> 3) & 0xFFFFFFu);
    const int w = (int)(key & 7u);
    if (w >= n || f >= (1ull << (n * n))) return MK_E_ARG;
    const int k = h_prog->nvars;
    bool exh = samples == 0 || k <= 1 || (k * n < 32 && (1ull << (k * n)) <= samples);
    if (!exh && !h_samples_n) return MK_E_ARG;
    if (!exh && j >= samples) return MK_E_ARG;
    const uint32_t x = exh ? j : h_samples_n[j];
    const uint32_t full = (1u << n) - 1u;
    std::memset(out, 0, sizeof(*out));
    out->phi = phi;
    out->psi = nullptr;
    out->n = (uint8_t)n;
    out->cls = (uint8_t)ci;
    out->world = (uint8_t)w;
    for (int v = 0; v < n; ++v) out->succ[v] = (uint32_t)((f >> (v * n)) & full);
    for (int i = 0; i < k; ++i) out->val[i] = (x >> (i * n)) & full;
    return MK_OK;
}
