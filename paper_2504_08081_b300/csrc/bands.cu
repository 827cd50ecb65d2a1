// Bandpass files (the paper's load_bandpass_from_file, Implementation,
// paragraph on bandpasses.py): a transmission curve read from text and, on
// request, resampled onto a uniform wavelength grid. Host code only.
//
// Format: one sample per line, wavelength then transmission, separated by
// blanks, tabs or a comma; further columns are ignored; '#' starts a comment;
// blank lines are skipped. Wavelengths are multiplied by wave_scale (e.g. 10
// for nanometres) and must be finite, positive and strictly ascending.
// Resampling treats the curve as piecewise linear between its samples (zero is
// not assumed outside): grid points are the multiples of `step` inside
// [first wavelength, last wavelength], each with the linear interpolant there.
#include <cerrno>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "salt_internal.cuh"

namespace {

int band_fail(salt_ctx *ctx, const std::string &msg) {
    if (ctx) {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->last_error = msg;
    }
    return SALT_ERR_INVALID;
}

// Parse the file into (wave, trans); returns an empty message on success.
std::string read_curve(const char *path, double wave_scale, std::vector<double> &w, std::vector<double> &t) {
    FILE *f = std::fopen(path, "r");
    if (!f) return std::string("cannot open ") + path + ": " + std::strerror(errno);
    std::string err;
    char line[4096];
    int ln = 0;
    while (std::fgets(line, sizeof line, f)) {
        ++ln;
        if (!std::strchr(line, '\n') && !std::feof(f)) {
            err = "line " + std::to_string(ln) + " is longer than 4095 characters";
            break;
        }
        if (char *h = std::strchr(line, '#')) *h = '\0';
        for (char *c = line; *c; ++c)
            if (*c == ',') *c = ' ';
        char *p = line;
        while (*p == ' ' || *p == '\t' || *p == '\r' || *p == '\n') ++p;
        if (!*p) continue;  // blank or comment-only line
        char *e1 = nullptr, *e2 = nullptr;
        const double lam = std::strtod(p, &e1);
        const double tr = (e1 && e1 != p) ? std::strtod(e1, &e2) : 0.0;
        if (!e1 || e1 == p || !e2 || e2 == e1) {
            err = "line " + std::to_string(ln) + ": expected a wavelength and a transmission";
            break;
        }
        const double wl = lam * wave_scale;
        if (!std::isfinite(wl) || !std::isfinite(tr) || !(wl > 0.0)) {
            err = "line " + std::to_string(ln) + ": non-finite or non-positive value";
            break;
        }
        if (!w.empty() && !(wl > w.back())) {
            err = "line " + std::to_string(ln) + ": wavelengths must be strictly ascending";
            break;
        }
        w.push_back(wl);
        t.push_back(tr);
    }
    std::fclose(f);
    if (err.empty() && w.size() < 2) err = std::string(path) + ": fewer than 2 samples";
    return err;
}

}  // namespace

extern "C" int salt_band_load(salt_ctx *ctx, const char *path, double wave_scale, double step, double *wave,
                              double *trans, int32_t capacity, int32_t *n) {
    if (!path || !n) return band_fail(ctx, "band file: missing path or count");
    if (!(wave_scale > 0.0) || !std::isfinite(wave_scale) || !(step >= 0.0) || !std::isfinite(step))
        return band_fail(ctx, "band file: wave_scale must be > 0 and step >= 0");
    std::vector<double> w, t;
    const std::string err = read_curve(path, wave_scale, w, t);
    if (!err.empty()) return band_fail(ctx, "band file: " + err);
    std::vector<double> ow, ot;
    if (step == 0.0) {
        ow = w;
        ot = t;
    } else {
        const double g0 = std::ceil(w.front() / step), g1 = std::floor(w.back() / step);
        if (!(g1 >= g0) || g1 - g0 > 1e7) return band_fail(ctx, "band file: step leaves no (or too many) samples");
        size_t seg = 0;
        for (double g = g0; g <= g1; g += 1.0) {
            const double x = g * step;
            while (seg + 2 < w.size() && w[seg + 1] < x) ++seg;  // w[seg] <= x <= w[seg+1]
            const double u = (x - w[seg]) / (w[seg + 1] - w[seg]);
            ow.push_back(x);
            ot.push_back(t[seg] + u * (t[seg + 1] - t[seg]));
        }
        if (ow.size() < 2) return band_fail(ctx, "band file: step leaves fewer than 2 samples");
    }
    if (ow.size() > (size_t)INT32_MAX) return band_fail(ctx, "band file: too many samples");
    *n = (int32_t)ow.size();
    if (!wave && !trans && capacity == 0) return SALT_OK;  // size query
    if (!wave || !trans || capacity < *n)
        return band_fail(ctx, "band file: output capacity " + std::to_string(capacity) + " < " +
                                  std::to_string(*n) + " samples");
    std::memcpy(wave, ow.data(), ow.size() * sizeof(double));
    std::memcpy(trans, ot.data(), ot.size() * sizeof(double));
    return SALT_OK;
}
