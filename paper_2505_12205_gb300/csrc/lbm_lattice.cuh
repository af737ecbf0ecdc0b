// Lattice descriptors of the phase-field WMRT lattice Boltzmann kernels.
//
// D3Q19: velocity order of the momentum rows 2-4 of eq:A2 (App. A), weights
// of eq:weights.  D2Q9: velocity order of the momentum rows 4 and 6 of eq:A1,
// standard weights 4/9, 1/9, 1/36 (the paper prints none for D2Q9).
//
// The WMRT collision (eq:mrt_collision with S-hat of eq:23) relaxes every
// moment at rate 1 except the deviatoric stress moments, which relax at s_nu.
// With M orthogonal under the weights W (eq:A2) -- or plainly orthogonal with
// equal weights on the support of the two stress rows (eq:A1) --
//     M^-1 S M = I - (1 - s_nu) P,   P = sum_k (W m_k)(m_k^T) / (m_k^T W m_k)
// over the stress rows k, so the collision needs only NS = 2 (D2Q9) or 5
// (D3Q19) dot products per node instead of a Q x Q matrix product.
#pragma once

namespace lbm {

struct D2Q9 {
    static constexpr int Q = 9;
    static constexpr int D = 2;
    static constexpr int NS = 2;           // stress moments relaxed at s_nu
    __host__ __device__ static constexpr int ex(int a)
    {
        constexpr int t[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
        return t[a];
    }
    __host__ __device__ static constexpr int ey(int a)
    {
        constexpr int t[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
        return t[a];
    }
    __host__ __device__ static constexpr int ez(int a)
    {
        constexpr int t[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
        return t[a];
    }
    __host__ __device__ static constexpr int opp(int a)
    {
        constexpr int t[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
        return t[a];
    }
    __host__ __device__ static constexpr float w(int a)
    {
        constexpr float t[9] = {4.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f, 1.f / 9.f,
                                   1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};
        return t[a];
    }
    // rows p_xx = e_x^2 - e_y^2 and p_xy = e_x e_y of eq:A1 (R5 reading: the
    // D2Q9 S-hat relaxes these two rows at s_nu)
    __host__ __device__ static constexpr int m(int k, int a)
    {
        return k == 0 ? ex(a) * ex(a) - ey(a) * ey(a) : ex(a) * ey(a);
    }
    // squared norms |m_k|^2 (4 and 4)
    __host__ __device__ static constexpr float norm(int k)
    {
        float s = 0.0f;
        for (int a = 0; a < Q; ++a) s += float(m(k, a) * m(k, a));
        return s;
    }
    // reconstruction weight of row k: unweighted orthogonality, m_k / |m_k|^2
    __host__ __device__ static constexpr float rw(int k, int a)
    {
        return float(m(k, a)) / norm(k);
    }
};

struct D3Q19 {
    static constexpr int Q = 19;
    static constexpr int D = 3;
    static constexpr int NS = 5;
    __host__ __device__ static constexpr int ex(int a)
    {
        constexpr int t[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
        return t[a];
    }
    __host__ __device__ static constexpr int ey(int a)
    {
        constexpr int t[19] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
        return t[a];
    }
    __host__ __device__ static constexpr int ez(int a)
    {
        constexpr int t[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};
        return t[a];
    }
    __host__ __device__ static constexpr int opp(int a)
    {
        constexpr int t[19] = {0, 2, 1, 4, 3, 6, 5, 8, 7, 10, 9, 12, 11, 14, 13, 16, 15, 18, 17};
        return t[a];
    }
    __host__ __device__ static constexpr float w(int a)
    {
        constexpr float t[19] = {12.f / 36.f, 2.f / 36.f, 2.f / 36.f, 2.f / 36.f, 2.f / 36.f,
                                    2.f / 36.f, 2.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f,
                                    1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f,
                                    1.f / 36.f, 1.f / 36.f, 1.f / 36.f, 1.f / 36.f};
        return t[a];
    }
    // rows 5-9 of eq:A2: e_x e_y, e_y e_z, e_x e_z, 2 e_x^2 - e_y^2 - e_z^2,
    // e_y^2 - e_z^2 (the entries relaxed at s_nu by eq:23)
    __host__ __device__ static constexpr int m(int k, int a)
    {
        return k == 0 ? ex(a) * ey(a)
             : k == 1 ? ey(a) * ez(a)
             : k == 2 ? ex(a) * ez(a)
             : k == 3 ? 2 * ex(a) * ex(a) - ey(a) * ey(a) - ez(a) * ez(a)
                      : ey(a) * ey(a) - ez(a) * ez(a);
    }
    // weighted norms m_k^T W m_k (1/9, 1/9, 1/9, 4/3, 4/9)
    __host__ __device__ static constexpr float norm(int k)
    {
        float s = 0.0f;
        for (int a = 0; a < Q; ++a) s += w(a) * float(m(k, a) * m(k, a));
        return s;
    }
    // reconstruction weight of row k: w_a m_ka / (m_k^T W m_k)
    __host__ __device__ static constexpr float rw(int k, int a)
    {
        return w(a) * float(m(k, a)) / norm(k);
    }
};

}  // namespace lbm
