// opcount.cpp -- the oracle's particle map, compiled with a counting double.
//
// TEST INFRASTRUCTURE ONLY: this measures the algorithmic floating-point work
// of the map as the oracle states it (section 2.2's step: two half kicks,
// each with the common term h0 and the direct terms of every planet, the
// Kepler drift solved to convergence, the encounter and escape tests).  It is
// used once, by oracle/opcount.py, on the 1024-particle workload; the product
// never links it.
//
// glisse_oracle.c is included as it is, with `double` replaced by cdouble, a
// value type that carries one double and counts every arithmetic operation
// applied to it: additions and subtractions, multiplications, divisions,
// square roots, and calls of transcendental functions (sin, cos, tan, atan2,
// sinh, cosh, atanh, cbrt), each as one operation; comparisons, fabs, floor
// and fmod are counted apart (they are not floating-point arithmetic in the
// usual FLOP count).  The results are those of the plain oracle bit for bit:
// cdouble does each operation in double, in the order written.  The
// complex-step tangent section of the oracle is left out of this build.
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <type_traits>
#ifdef _OPENMP
#include <omp.h>
#endif

namespace opcount {
struct Counts {
    uint64_t add, mul, div, sqrt, trans, cmp, other;
};
static Counts g;  // the counting run is single-threaded
}  // namespace opcount

struct cdouble {
    double v;
    cdouble() = default;
    cdouble(double x) : v(x) {}
    explicit operator double() const { return v; }
    explicit operator bool() const { return v != 0.0; }
    cdouble& operator+=(cdouble b) { ++opcount::g.add; v += b.v; return *this; }
    cdouble& operator-=(cdouble b) { ++opcount::g.add; v -= b.v; return *this; }
    cdouble& operator*=(cdouble b) { ++opcount::g.mul; v *= b.v; return *this; }
    cdouble& operator/=(cdouble b) { ++opcount::g.div; v /= b.v; return *this; }
    cdouble operator-() const { return cdouble(-v); }  // a sign flip, not counted
    cdouble operator+() const { return *this; }
};
static_assert(std::is_trivially_copyable<cdouble>::value && sizeof(cdouble) == sizeof(double), "layout");

template <class T>
using if_arith = typename std::enable_if<std::is_arithmetic<T>::value, int>::type;

// binary arithmetic: cdouble with cdouble, and with any built-in arithmetic type on either side
#define OPC_BINARY(OP, FIELD)                                                                               \
    inline cdouble operator OP(cdouble a, cdouble b) { ++opcount::g.FIELD; return cdouble(a.v OP b.v); }     \
    template <class T, if_arith<T> = 0>                                                                      \
    inline cdouble operator OP(cdouble a, T b) { ++opcount::g.FIELD; return cdouble(a.v OP(double) b); }     \
    template <class T, if_arith<T> = 0>                                                                      \
    inline cdouble operator OP(T a, cdouble b) { ++opcount::g.FIELD; return cdouble((double)a OP b.v); }
OPC_BINARY(+, add)
OPC_BINARY(-, add)
OPC_BINARY(*, mul)
OPC_BINARY(/, div)
#undef OPC_BINARY

#define OPC_COMPARE(OP)                                                                              \
    inline bool operator OP(cdouble a, cdouble b) { ++opcount::g.cmp; return a.v OP b.v; }            \
    template <class T, if_arith<T> = 0>                                                               \
    inline bool operator OP(cdouble a, T b) { ++opcount::g.cmp; return a.v OP(double) b; }            \
    template <class T, if_arith<T> = 0>                                                               \
    inline bool operator OP(T a, cdouble b) { ++opcount::g.cmp; return (double)a OP b.v; }
OPC_COMPARE(<)
OPC_COMPARE(>)
OPC_COMPARE(<=)
OPC_COMPARE(>=)
OPC_COMPARE(==)
OPC_COMPARE(!=)
#undef OPC_COMPARE

inline cdouble sqrt(cdouble x) { ++opcount::g.sqrt; return cdouble(::sqrt(x.v)); }
#define OPC_TRANS1(F) \
    inline cdouble F(cdouble x) { ++opcount::g.trans; return cdouble(::F(x.v)); }
OPC_TRANS1(sin)
OPC_TRANS1(cos)
OPC_TRANS1(tan)
OPC_TRANS1(sinh)
OPC_TRANS1(cosh)
OPC_TRANS1(atanh)
OPC_TRANS1(cbrt)
#undef OPC_TRANS1
inline cdouble atan2(cdouble y, cdouble x) { ++opcount::g.trans; return cdouble(::atan2(y.v, x.v)); }
inline cdouble fabs(cdouble x) { ++opcount::g.other; return cdouble(::fabs(x.v)); }
inline cdouble floor(cdouble x) { ++opcount::g.other; return cdouble(::floor(x.v)); }
inline cdouble fmod(cdouble x, cdouble y) { ++opcount::g.other; return cdouble(::fmod(x.v, y.v)); }
inline bool isfinite(cdouble x) { return std::isfinite(x.v); }

#define ORC_OPCOUNT 1
#define _Thread_local thread_local
#define double cdouble
#include "glisse_oracle.c"
#undef double
#undef _Thread_local

// The particle map of orc_particles_ex over a given planet log, counting operations.
// Arguments as orc_particles_ex (plain doubles; converted in and out), one thread.
// counts: out [7] additions, multiplications, divisions, square roots,
// transcendental calls, comparisons, other (fabs, floor, fmod) over the whole run.
extern "C" int orc_opcount_particles(double m0, int np, const double* pmass, const double* log_pos, int64_t nsteps,
                                     double dt, const double* rcrit, double rmax, double* state, int64_t npart,
                                     int64_t* removal_step, int32_t* reason, uint64_t* counts) {
    const size_t nlog = (size_t)(nsteps + 1) * 3 * (size_t)(np > 0 ? np : 1);
    cdouble* lg = (cdouble*)malloc(sizeof(cdouble) * nlog);
    cdouble* st = (cdouble*)malloc(sizeof(cdouble) * 6 * (size_t)(npart > 0 ? npart : 1));
    cdouble* mg = (cdouble*)malloc(sizeof(cdouble) * (size_t)(npart > 0 ? npart : 1));
    cdouble* cl = (cdouble*)malloc(sizeof(cdouble) * (size_t)(npart > 0 ? npart : 1));
    cdouble pm[ORC_MAXP], rc[ORC_MAXP];
    if (!lg || !st || !mg || !cl || np > ORC_MAXP) {
        free(lg), free(st), free(mg), free(cl);
        return ORC_EINVAL;
    }
    for (size_t i = 0; i < (size_t)(nsteps + 1) * 3 * (size_t)np; ++i) lg[i] = log_pos[i];
    for (int64_t i = 0; i < 6 * npart; ++i) st[i] = state[i];
    for (int64_t i = 0; i < npart; ++i) {
        mg[i] = HUGE_VAL;
        cl[i] = HUGE_VAL;
        removal_step[i] = -1;
        reason[i] = 0;
    }
    for (int j = 0; j < np; ++j) {
        pm[j] = pmass[j];
        rc[j] = rcrit[j];
    }
    opcount::g = opcount::Counts{};
    const int rcode = orc_particles_ex(cdouble(m0), np, pm, lg, nsteps, cdouble(dt), rc, cdouble(rmax), st, npart,
                                       removal_step, reason, mg, cl, 0, 1, 1, 0, cdouble(0.0), nullptr);
    const opcount::Counts c = opcount::g;
    counts[0] = c.add;
    counts[1] = c.mul;
    counts[2] = c.div;
    counts[3] = c.sqrt;
    counts[4] = c.trans;
    counts[5] = c.cmp;
    counts[6] = c.other;
    for (int64_t i = 0; i < 6 * npart; ++i) state[i] = st[i].v;
    free(lg), free(st), free(mg), free(cl);
    return rcode;
}
