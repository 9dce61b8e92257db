// QAPLIB text layout: reading instances, reading and writing solutions.
// Host code only (no device work).
//
// Instance file: the size n, then the n x n matrix A, then the n x n matrix
// B, as whitespace-separated decimal integers; rows may wrap across lines and
// blank lines may appear anywhere. The objective of such a file is
// sum_ij A_ij B_{p(i)p(j)}, which is Eq. 1 with D = A and F = B.
// Solution file: "n cost", then the n entries of p, 1-based.
#include <cerrno>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../../include/pdit.h"

namespace {

// Whitespace-separated decimal integer reader over a FILE*.
struct TokenReader {
    FILE *f;
    // 1: read a value; 0: end of file; -1: malformed token or out of int64 range.
    int next(long long *out) {
        int c;
        do {
            c = std::fgetc(f);
        } while (c == ' ' || c == '\t' || c == '\n' || c == '\r' || c == '\f' || c == '\v');
        if (c == EOF) return 0;
        char buf[32];
        int len = 0;
        while (c != EOF && !(c == ' ' || c == '\t' || c == '\n' || c == '\r' || c == '\f' || c == '\v')) {
            if (len + 1 >= (int)sizeof(buf)) return -1;
            buf[len++] = (char)c;
            c = std::fgetc(f);
        }
        buf[len] = '\0';
        char *end = nullptr;
        errno = 0;
        const long long v = std::strtoll(buf, &end, 10);
        if (errno != 0 || end == buf || *end != '\0') return -1;
        *out = v;
        return 1;
    }
};

struct File {
    FILE *f;
    explicit File(FILE *fp) : f(fp) {}
    ~File() {
        if (f) std::fclose(f);
    }
};

bool in_int32(long long v) { return v >= -2147483648ll && v <= 2147483647ll; }

}  // namespace

extern "C" {

int pdit_read_qaplib(const char *path, int *n, int32_t *D, int32_t *F, size_t capacity) {
    if (!path || !n) return PDIT_EINVAL;
    *n = 0;
    File file(std::fopen(path, "r"));
    if (!file.f) return PDIT_EIO;
    TokenReader rd{file.f};
    long long v = 0;
    if (rd.next(&v) != 1) return PDIT_EINVAL;
    if (v < 2 || v > PDIT_N_MAX) return PDIT_EINVAL;
    const int size = (int)v;
    const size_t nn = (size_t)size * size;
    const bool fill = D != nullptr || F != nullptr;
    if (fill && (!D || !F)) return PDIT_EINVAL;
    if (fill && capacity < nn) return PDIT_ENOMEM;
    for (int m = 0; m < 2; ++m) {
        int32_t *dst = m == 0 ? D : F;
        for (size_t k = 0; k < nn; ++k) {
            if (rd.next(&v) != 1 || !in_int32(v)) return PDIT_EINVAL;
            if (fill) dst[k] = (int32_t)v;
        }
    }
    if (rd.next(&v) != 0) return PDIT_EINVAL;  // trailing tokens
    *n = size;
    return PDIT_OK;
}

int pdit_read_qaplib_solution(const char *path, int *n, int64_t *cost, int32_t *perm, int capacity) {
    if (!path || !n || !cost) return PDIT_EINVAL;
    *n = 0;
    File file(std::fopen(path, "r"));
    if (!file.f) return PDIT_EIO;
    TokenReader rd{file.f};
    long long v = 0, c = 0;
    if (rd.next(&v) != 1 || v < 2 || v > PDIT_N_MAX) return PDIT_EINVAL;
    const int size = (int)v;
    if (rd.next(&c) != 1) return PDIT_EINVAL;
    if (perm && capacity < size) return PDIT_ENOMEM;
    unsigned char seen[PDIT_N_MAX] = {};
    for (int k = 0; k < size; ++k) {
        if (rd.next(&v) != 1 || v < 1 || v > size || seen[v - 1]) return PDIT_EINVAL;
        seen[v - 1] = 1;
        if (perm) perm[k] = (int32_t)(v - 1);
    }
    if (rd.next(&v) != 0) return PDIT_EINVAL;
    *n = size;
    *cost = (int64_t)c;
    return PDIT_OK;
}

int pdit_write_qaplib_solution(const char *path, int n, int64_t cost, const int32_t *perm) {
    if (!path || !perm || n < 2 || n > PDIT_N_MAX) return PDIT_EINVAL;
    unsigned char seen[PDIT_N_MAX] = {};
    for (int k = 0; k < n; ++k) {
        if (perm[k] < 0 || perm[k] >= n || seen[perm[k]]) return PDIT_EINVAL;
        seen[perm[k]] = 1;
    }
    File file(std::fopen(path, "w"));
    if (!file.f) return PDIT_EIO;
    bool ok = std::fprintf(file.f, "%d %lld\n", n, (long long)cost) > 0;
    for (int k = 0; ok && k < n; ++k) ok = std::fprintf(file.f, k + 1 < n ? "%d " : "%d\n", perm[k] + 1) > 0;
    if (std::fflush(file.f) != 0) ok = false;
    return ok ? PDIT_OK : PDIT_EIO;
}

}  // extern "C"
