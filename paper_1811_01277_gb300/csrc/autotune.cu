// Autotuning of the back-transformation's kernel choice and blocking,
// modelled on the paper's autotuning (Sec. 4.3): a tuning object walks a
// fixed list of settings, the caller runs one solve (here: one
// back-transformation) per setting and reports how long it took, and at the
// end the fastest setting is kept.  The walk can be saved to a text file and
// resumed, so that it can be spread over the iterations of an application's
// self-consistency loop (Sec. 5.3).
//   FAST   : the kernel variant only (wavefront, pipeline, tensor-core pipeline)
//   MEDIUM : the variant and its blocking (sweeps per tile, columns per block;
//            column batch for the tensor-core pipeline)
// Host code only; no device memory is touched.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <vector>

#include "elpa_gb300.h"

struct gb_autotune {
    int level, n, nbw, nev;
    std::vector<gb_trans_ev_opts> cand;
    std::vector<double> secs;  // < 0: not measured yet
    int next;                  // index of the next candidate to hand out
    int pending;               // candidate handed out and not yet reported (-1: none)
};

namespace {

bool pipeline_ok(int nbw) { return nbw == 8 || nbw == 16 || nbw == 32 || nbw == 64; }
bool tc_ok(int nbw) { return nbw == 16 || nbw == 32 || nbw == 64; }

void build_candidates(gb_autotune *t)
{
    t->cand.clear();
    auto add = [&](int variant, int nb, int cols, int batch = 0) {
        gb_trans_ev_opts o;
        memset(&o, 0, sizeof(o));
        o.variant = variant;
        o.sweeps_per_tile = nb;
        o.cols_per_block = cols;
        o.column_batch = batch;
        t->cand.push_back(o);
    };
    const bool real_reg = t->nbw <= 64;
    if (t->level == GB_AUTOTUNE_FAST) {
        add(GB_VARIANT_WAVEFRONT, 0, 0);
        if (pipeline_ok(t->nbw)) add(GB_VARIANT_PIPELINE, 0, 0);
        if (tc_ok(t->nbw)) add(GB_VARIANT_PIPELINE_TC, 0, 0);
        if (tc_ok(t->nbw)) add(GB_VARIANT_PIPELINE_TC5, 0, 0);
    } else {
        const int wnb[3] = {4, 8, 16}, wcols[3] = {32, 64, 128};
        for (int a = 0; a < 3; a++)
            for (int c = 0; c < 3; c++)
                if (real_reg || wcols[c] <= 64) add(GB_VARIANT_WAVEFRONT, wnb[a], wcols[c]);
        if (pipeline_ok(t->nbw)) {
            const int pnb[2] = {8, 16}, pcols[2] = {64, 128};
            for (int a = 0; a < 2; a++)
                for (int c = 0; c < 2; c++) add(GB_VARIANT_PIPELINE, pnb[a], pcols[c]);
        }
        if (tc_ok(t->nbw)) {
            const int tcb[3] = {8, 16, 32};
            for (int a = 0; a < 3; a++) add(GB_VARIANT_PIPELINE_TC, 0, 0, tcb[a]);
            const int tc5b[3] = {2, 4, 8};  // 128-column blocks per batch
            for (int a = 0; a < 3; a++) add(GB_VARIANT_PIPELINE_TC5, 0, 0, tc5b[a]);
        }
    }
    t->secs.assign(t->cand.size(), -1.0);
}

}  // namespace

extern "C" {

gb_autotune *gb_autotune_create(int level, int n, int nbw, int nev)
{
    if ((level != GB_AUTOTUNE_FAST && level != GB_AUTOTUNE_MEDIUM) || n < 1 || nbw < 1 || nev < 0) return NULL;
    gb_autotune *t = new gb_autotune;
    t->level = level;
    t->n = n;
    t->nbw = nbw;
    t->nev = nev;
    t->next = 0;
    t->pending = -1;
    build_candidates(t);
    return t;
}

void gb_autotune_destroy(gb_autotune *t) { delete t; }

int gb_autotune_step(gb_autotune *t, gb_trans_ev_opts *next)
{
    if (!t) return -1;
    if (!next) return -2;
    if (t->pending >= 0) return -1;  // report the previous candidate first
    if (t->next >= (int)t->cand.size()) return 0;
    *next = t->cand[t->next];
    t->pending = t->next++;
    return 1;
}

int gb_autotune_report(gb_autotune *t, double seconds)
{
    if (!t || t->pending < 0) return -1;
    if (!(seconds >= 0.0)) return -2;
    t->secs[t->pending] = seconds;
    t->pending = -1;
    return 0;
}

int gb_autotune_best(const gb_autotune *t, gb_trans_ev_opts *best, double *seconds)
{
    if (!t) return -1;
    if (!best) return -2;
    int bi = -1;
    for (size_t i = 0; i < t->secs.size(); i++)
        if (t->secs[i] >= 0.0 && (bi < 0 || t->secs[i] < t->secs[bi])) bi = (int)i;
    if (bi < 0) return GB_ERR_UNSUPPORTED;  // nothing measured yet
    *best = t->cand[bi];
    if (seconds) *seconds = t->secs[bi];
    return GB_OK;
}

int gb_autotune_progress(const gb_autotune *t, int *tried, int *total)
{
    if (!t) return -1;
    if (tried) *tried = t->next;
    if (total) *total = (int)t->cand.size();
    return GB_OK;
}

int gb_autotune_save(const gb_autotune *t, const char *path)
{
    if (!t) return -1;
    if (!path) return -2;
    FILE *f = fopen(path, "w");
    if (!f) return GB_ERR_UNSUPPORTED;
    // a candidate handed out but not reported yet is tried again on resume
    const int next = t->pending >= 0 ? t->pending : t->next;
    fprintf(f, "gb_autotune 2\nlevel %d\nn %d\nnbw %d\nnev %d\nnext %d\ncandidates %zu\n", t->level, t->n, t->nbw,
            t->nev, next, t->cand.size());
    for (size_t i = 0; i < t->cand.size(); i++)
        fprintf(f, "c %d %d %d %d %.17g\n", t->cand[i].variant, t->cand[i].sweeps_per_tile, t->cand[i].cols_per_block,
                t->cand[i].column_batch, t->secs[i]);
    int rc = fclose(f);
    return rc == 0 ? GB_OK : GB_ERR_UNSUPPORTED;
}

gb_autotune *gb_autotune_load(const char *path)
{
    if (!path) return NULL;
    FILE *f = fopen(path, "r");
    if (!f) return NULL;
    int ver = 0, level = 0, n = 0, nbw = 0, nev = 0, next = 0;
    size_t ncand = 0;
    gb_autotune *t = NULL;
    if (fscanf(f, "gb_autotune %d level %d n %d nbw %d nev %d next %d candidates %zu", &ver, &level, &n, &nbw, &nev,
               &next, &ncand) == 7 &&
        ver == 2) {
        t = gb_autotune_create(level, n, nbw, nev);
        if (t && ncand == t->cand.size() && next >= 0 && next <= (int)ncand) {
            for (size_t i = 0; i < ncand; i++) {
                int v, nb, cols, cb;
                double s;
                if (fscanf(f, " c %d %d %d %d %lg", &v, &nb, &cols, &cb, &s) != 5 || v != t->cand[i].variant ||
                    nb != t->cand[i].sweeps_per_tile || cols != t->cand[i].cols_per_block ||
                    cb != t->cand[i].column_batch) {
                    delete t;
                    t = NULL;
                    break;
                }
                t->secs[i] = s;
            }
            if (t) t->next = next;
        } else if (t) {
            delete t;
            t = NULL;
        }
    }
    fclose(f);
    return t;
}

}  // extern "C"

// Band-width tuning of the two-stage solve by size class (declared in
// elpa_gb300.h): the same walk-and-report protocol, over (n, nbw) trials.
struct gb_solve_tuner {
    int n_lo, n_hi, classes;
    struct Trial {
        int cls, n, nbw;
        double secs;  // < 0: not measured yet
    };
    std::vector<Trial> trials;
    int next, pending;
};

namespace {

// class c covers [n_lo r^c, n_lo r^(c+1)), r = (n_hi / n_lo)^(1 / classes);
// n_hi itself belongs to the last class
int tuner_class(const gb_solve_tuner *t, int n)
{
    if (n < t->n_lo || n > t->n_hi) return -1;
    if (t->n_hi == t->n_lo) return 0;
    const double x = log((double)n / t->n_lo) / log((double)t->n_hi / t->n_lo) * t->classes;
    int c = (int)floor(x);
    return c < 0 ? 0 : (c >= t->classes ? t->classes - 1 : c);
}

void tuner_trials(gb_solve_tuner *t)
{
    t->trials.clear();
    const double r = t->n_hi == t->n_lo ? 1.0 : pow((double)t->n_hi / t->n_lo, 1.0 / t->classes);
    for (int c = 0; c < t->classes; c++) {
        int n = (int)lround(t->n_lo * pow(r, c + 0.5));
        n = n < t->n_lo ? t->n_lo : (n > t->n_hi ? t->n_hi : n);
        const int cand[3] = {16, 32, 64};
        bool any = false;
        for (int b : cand)
            if (b < n) {
                t->trials.push_back({c, n, b, -1.0});
                any = true;
            }
        if (!any) t->trials.push_back({c, n, n - 1, -1.0});
    }
}

}  // namespace

extern "C" {

gb_solve_tuner *gb_solve_tuner_create(int n_lo, int n_hi, int classes)
{
    if (n_lo < 2 || n_hi < n_lo || classes < 1 || classes > 64) return NULL;
    gb_solve_tuner *t = new gb_solve_tuner;
    t->n_lo = n_lo;
    t->n_hi = n_hi;
    t->classes = classes;
    t->next = 0;
    t->pending = -1;
    tuner_trials(t);
    return t;
}

void gb_solve_tuner_destroy(gb_solve_tuner *t) { delete t; }

int gb_solve_tuner_step(gb_solve_tuner *t, int *n, int *nbw)
{
    if (!t) return -1;
    if (!n || !nbw) return -2;
    if (t->pending >= 0) return -1;
    if (t->next >= (int)t->trials.size()) return 0;
    *n = t->trials[t->next].n;
    *nbw = t->trials[t->next].nbw;
    t->pending = t->next++;
    return 1;
}

int gb_solve_tuner_report(gb_solve_tuner *t, double seconds)
{
    if (!t || t->pending < 0) return -1;
    if (!(seconds >= 0.0)) return -2;
    t->trials[t->pending].secs = seconds;
    t->pending = -1;
    return 0;
}

int gb_solve_tuner_nbw(const gb_solve_tuner *t, int n)
{
    if (n < 2) return -1;
    const int c = t ? tuner_class(t, n) : -1;
    int best = -1;
    double bs = 0.0;
    if (c >= 0)
        for (const auto &tr : t->trials)
            if (tr.cls == c && tr.secs >= 0.0 && (best < 0 || tr.secs < bs)) {
                best = tr.nbw;
                bs = tr.secs;
            }
    if (best < 0) return gb_solve_default_nbw(n);
    return best < n ? best : n - 1;
}

int gb_solve_tuner_save(const gb_solve_tuner *t, const char *path)
{
    if (!t) return -1;
    if (!path) return -2;
    FILE *f = fopen(path, "w");
    if (!f) return GB_ERR_UNSUPPORTED;
    const int next = t->pending >= 0 ? t->pending : t->next;
    fprintf(f, "gb_solve_tuner 1\nn_lo %d\nn_hi %d\nclasses %d\nnext %d\ntrials %zu\n", t->n_lo, t->n_hi, t->classes,
            next, t->trials.size());
    for (const auto &tr : t->trials) fprintf(f, "t %d %d %d %.17g\n", tr.cls, tr.n, tr.nbw, tr.secs);
    return fclose(f) == 0 ? GB_OK : GB_ERR_UNSUPPORTED;
}

gb_solve_tuner *gb_solve_tuner_load(const char *path)
{
    if (!path) return NULL;
    FILE *f = fopen(path, "r");
    if (!f) return NULL;
    int ver = 0, lo = 0, hi = 0, classes = 0, next = 0;
    size_t nt = 0;
    gb_solve_tuner *t = NULL;
    if (fscanf(f, "gb_solve_tuner %d n_lo %d n_hi %d classes %d next %d trials %zu", &ver, &lo, &hi, &classes, &next,
               &nt) == 6 &&
        ver == 1 && (t = gb_solve_tuner_create(lo, hi, classes)) != NULL) {
        bool ok = nt == t->trials.size() && next >= 0 && next <= (int)nt;
        for (size_t i = 0; ok && i < nt; i++) {
            int c, n, b;
            double s;
            ok = fscanf(f, " t %d %d %d %lg", &c, &n, &b, &s) == 4 && c == t->trials[i].cls && n == t->trials[i].n &&
                 b == t->trials[i].nbw;
            if (ok) t->trials[i].secs = s;
        }
        if (ok) {
            t->next = next;
        } else {
            delete t;
            t = NULL;
        }
    }
    fclose(f);
    return t;
}

}  // extern "C"
