"""Hand-built tiny scenes for closed-form pins (test fixtures only)."""
import numpy as np

from paper_1702_01530_gb300 import scenegen as sg


def scene(spheres=(), tris=(), mats=((0.5, 0.5, 0.5, 0.0),), lights=(((0.0, 10.0, 0.0), 1.0),),
          eye=(0, 0, 0), forward=(0, 0, -1), up=(0, 1, 0), vfov=60.0, W=33, H=33,
          eye_sep=0.0, convergence=10.0, max_depth=3, name="hand"):
    """spheres: ((cx,cy,cz), r, mat); tris: (v0, v1, v2, mat); mats: (r,g,b,refl)."""
    sp = np.zeros(len(spheres), sg.SPHERE_DT)
    for k, (c, r, m) in enumerate(spheres):
        sp[k]["center"], sp[k]["radius"], sp[k]["material"] = c, r, m
    tr = np.zeros(len(tris), sg.TRIANGLE_DT)
    for k, (a, b, c, m) in enumerate(tris):
        tr[k]["v0"], tr[k]["v1"], tr[k]["v2"], tr[k]["material"] = a, b, c, m
    mt = np.zeros(len(mats), sg.MATERIAL_DT)
    for k, (r, g, b, refl) in enumerate(mats):
        mt[k]["albedo"], mt[k]["reflectivity"] = (r, g, b), refl
    li = np.zeros(len(lights), sg.LIGHT_DT)
    for k, (p, inten) in enumerate(lights):
        li[k]["position"], li[k]["intensity"] = p, inten
    cam = sg.make_camera(eye, forward, up, vfov)
    return sg.Scene(name, sp, tr, mt, li, cam, eye_sep, convergence, W, H, max_depth)


def quad(x0, x1, y0, y1, z, mat):
    """Two triangles covering [x0,x1] x [y0,y1] in the plane z."""
    a, b, c, d = (x0, y0, z), (x1, y0, z), (x1, y1, z), (x0, y1, z)
    return [(a, b, c, mat), (a, c, d, mat)]


def quad_xz(x0, x1, z0, z1, y, mat):
    a, b, c, d = (x0, y, z0), (x1, y, z0), (x1, y, z1), (x0, y, z1)
    return [(a, b, c, mat), (a, c, d, mat)]
