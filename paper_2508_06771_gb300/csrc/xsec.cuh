// xsec.cuh -- tabulated cross sections of the electron-neutral step.
//
// Sec. 4.2 evaluates each cross section as a piecewise polynomial instead of
// looking it up in a table.  Layout (set by ltpc_set_cross_sections): interval
// i of a uniform grid in ln E, ln E0 + [i, i+1) h, holds a cubic
// c0 + c1 t + c2 t^2 + c3 t^3 in t = (ln E - ln E0)/h - i; below E0 the value is
// 0 (zero_below, as an ionization threshold) or the first knot's, above the
// last knot the last knot's.  binary64 follows the reference's operations
// (natural log, one division, Horner); binary32 uses the SFU logarithm and a
// binary32 copy of the coefficients.
#pragma once
#include <stdint.h>

namespace ltpc {

constexpr int XS_MAX_PIECES = 256;

struct XsTable {
    int32_t pieces;          // 0: no table (constant / step cross section)
    int32_t zero_below;
    double lnE0, h;
    float lnE0f, inv_hf;
    const double* cd;        // [pieces][4] device
    const float* cf;         // [pieces][4] device, binary32 copy
};

struct XsArgs {
    XsTable el, ion;
    int32_t on;              // 1: sigma_el / sigma_ion from the tables
    int32_t per_particle;    // 1: per-particle collision probabilities instead of null collisions
};

template <class T> struct XsEval;
template <> struct XsEval<double> {
    static __device__ __forceinline__ double eval(const XsTable& t, double E)
    {
        if (!(E > 0.0)) return t.zero_below ? 0.0 : __ldg(t.cd);
        const double u = (log(E) - t.lnE0) / t.h;
        if (u < 0.0) return t.zero_below ? 0.0 : __ldg(t.cd);
        const double fi = floor(u);
        int32_t i = (int32_t)fi;
        double x;
        if (i >= t.pieces) { i = t.pieces - 1; x = 1.0; }
        else x = u - fi;
        const double* c = t.cd + 4 * i;
        return __ldg(c) + x * (__ldg(c + 1) + x * (__ldg(c + 2) + x * __ldg(c + 3)));
    }
};
template <> struct XsEval<float> {
    static __device__ __forceinline__ float eval(const XsTable& t, float E)
    {
        if (!(E > 0.0f)) return t.zero_below ? 0.0f : __ldg(t.cf);
        const float u = (__logf(E) - t.lnE0f) * t.inv_hf;
        if (u < 0.0f) return t.zero_below ? 0.0f : __ldg(t.cf);
        const float fi = floorf(u);
        int32_t i = (int32_t)fi;
        float x;
        if (i >= t.pieces) { i = t.pieces - 1; x = 1.0f; }
        else x = u - fi;
        const float4 c = __ldg(reinterpret_cast<const float4*>(t.cf) + i);
        return c.x + x * (c.y + x * (c.z + x * c.w));
    }
};

// sigma_el(E) and sigma_ion(E): the tables when on, else the constants (the
// ionization one above its threshold).
template <class T>
__device__ __forceinline__ T xs_el(const XsArgs& x, T E, T sig_el)
{
    return x.on && x.el.pieces ? XsEval<T>::eval(x.el, E) : sig_el;
}
template <class T>
__device__ __forceinline__ T xs_ion(const XsArgs& x, T E, T sig_ion, T e_ion)
{
    if (x.on && x.ion.pieces) return XsEval<T>::eval(x.ion, E);
    return E >= e_ion ? sig_ion : T(0);
}

}  // namespace ltpc
