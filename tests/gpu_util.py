"""Helpers shared by the GPU parity tests (CUDA path vs oracle)."""
import numpy as np

import oracle as orc
import paper_2406_06963_b300 as dhrs


def trace_gpu(scene, cam, params, precision=dhrs.DHR_FP32):
    import torch
    g = dhrs.GBuffer(cam.width, cam.height, precision)
    mask = torch.empty((cam.height, cam.width), dtype=torch.uint8, device="cuda")
    ao = torch.empty_like(mask)
    dhrs.trace_visibility(scene, cam, params, g, mask, ao)
    torch.cuda.synchronize()
    zn = g.to_fp32().depth_normal.cpu().numpy().reshape(-1, 4)
    return dict(depth=zn[:, 0].astype(np.float64), normal=zn[:, 1:].astype(np.float64),
                mesh=g.mesh_u32().ravel(), shadow_mask=mask.cpu().numpy().ravel(),
                ao_count=ao.cpu().numpy().ravel(), gbuf=g, mask_t=mask, ao_t=ao)


def gpu_params(tp: "orc.TraceParams"):
    return dhrs.TraceParams(light_dirs=tp.light_dirs, cone_half_angle_deg=tp.cone_half_angle_deg,
                            ao_radius=tp.ao_radius, ao_spp=tp.ao_spp, frame=tp.frame, seed=tp.seed)


def compare_trace(gpu, ref, idx, n_lights, ao_spp):
    """Compare GPU outputs at flat pixel indices `idx` with the oracle's
    results for the same pixels.  Returns a dict of counts; disagreements
    that the oracle did not flag as within its grazing margin are listed in
    'unexplained'."""
    g_mesh = gpu["mesh"][idx]
    r_mesh = ref["mesh"]
    amb_p = ref["amb_primary"].astype(bool)
    prim_bad = g_mesh != r_mesh
    res = dict(pixels=len(idx), primary_disagree=int(prim_bad.sum()),
               primary_unexplained=int((prim_bad & ~amb_p).sum()))
    same = ~prim_bad & (r_mesh != 0xFFFFFFFF) & ~amb_p
    dz = np.abs(gpu["depth"][idx][same] - ref["depth"][same]) / np.maximum(ref["depth"][same], 1e-6)
    dn = np.abs(gpu["normal"][idx][same] - ref["normal"][same]).max(1) if same.any() else np.zeros(0)
    res["depth_rel_max"] = float(dz.max()) if dz.size else 0.0
    res["normal_abs_max"] = float(dn.max()) if dn.size else 0.0
    ok = ~prim_bad & ~amb_p
    # shadow bits
    sh_bad = 0
    sh_unexp = 0
    for k in range(n_lights):
        gb = (gpu["shadow_mask"][idx] >> k) & 1
        rb = (ref["shadow_mask"] >> k) & 1
        ab = (ref["amb_shadow"] >> k) & 1
        bad = ok & (gb != rb)
        sh_bad += int(bad.sum())
        sh_unexp += int((bad & (ab == 0)).sum())
    # AO counts: a difference may not exceed the number of ambiguous AO rays
    dao = np.abs(gpu["ao_count"][idx].astype(int) - ref["ao_count"].astype(int))
    ao_bad = int(dao[ok].sum())
    ao_unexp = int((ok & (dao > ref["amb_ao"])).sum())
    res.update(shadow_disagree=sh_bad, shadow_unexplained=sh_unexp, ao_disagree=ao_bad,
               ao_unexplained=ao_unexp)
    fg = r_mesh != 0xFFFFFFFF
    n_rays = len(idx) + int(fg.sum()) * (n_lights + ao_spp)
    res["rays"] = n_rays
    res["disagree"] = res["primary_disagree"] + sh_bad + ao_bad
    res["disagree_frac"] = res["disagree"] / max(1, n_rays)
    res["ambiguous_rays"] = int(amb_p.sum()) + int(sum(bin(int(a)).count("1") for a in ref["amb_shadow"])) \
        + int(ref["amb_ao"].sum())
    return res
