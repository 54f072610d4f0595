"""Seeded analytic scenes and their flat float32 description ("scene blob").

Scene blob layout (float32, read independently by the CUDA library and by the
oracle -- it is a file format, not shared code):

  header (HEADER_LEN = 48 floats)
    [0] n_spheres  [1] n_boxes  [2] has_room (1/0)  [3] rotating sphere index (-1: none)
    [4:7] room_min  [7:10] room_max
    [10:13] sky radiance RGB (seen through the skylight, or everywhere if no room)
    [13:17] skylight opening in the +y wall: x0, x1, z0, z1 (none if x0 >= x1)
    [17] wall emitted radiance (grey, all six walls; furnace scenes only)
    [18:36] wall albedo RGB for the walls -x, +x, -y, +y, -z, +z
    [36:39] point on the vertical (+y) rotation axis of the rotating sphere
    [39:48] reserved (0)
  spheres, SPHERE_LEN = 12 floats each:
    centre xyz, radius, albedo RGB, emitted radiance RGB, 0, 0
  boxes, BOX_LEN = 12 floats each:
    min xyz, max xyz, albedo RGB, 0, 0, 0

All surfaces are Lambertian; the room is the inside of an axis-aligned box.
"""
import math
from dataclasses import dataclass, field

import numpy as np

HEADER_LEN = 48
SPHERE_LEN = 12
BOX_LEN = 12

ROOM_MIN = (-5.0, -5.0, -5.0)
ROOM_MAX = (5.0, 5.0, 5.0)
CAMERA_POS = (0.0, 0.0, -4.9)
EMITTER_CENTRE = (3.0, 3.0, 0.0)
EMITTER_RADIUS = 0.5
EMITTER_RADIANCE = 20.0
SKYLIGHT = (-2.0, 2.0, -2.0, 2.0)
WALL_ALBEDO = (
    (0.75, 0.25, 0.25),  # -x
    (0.25, 0.75, 0.25),  # +x
    (0.70, 0.70, 0.70),  # -y (floor)
    (0.80, 0.80, 0.80),  # +y (ceiling)
    (0.70, 0.70, 0.70),  # -z
    (0.60, 0.60, 0.75),  # +z
)


@dataclass
class Scene:
    spheres: np.ndarray = field(default_factory=lambda: np.zeros((0, SPHERE_LEN), np.float32))
    boxes: np.ndarray = field(default_factory=lambda: np.zeros((0, BOX_LEN), np.float32))
    has_room: bool = False
    room_min: tuple = ROOM_MIN
    room_max: tuple = ROOM_MAX
    sky: tuple = (0.0, 0.0, 0.0)
    skylight: tuple = (0.0, 0.0, 0.0, 0.0)
    wall_emission: float = 0.0
    wall_albedo: tuple = WALL_ALBEDO
    rot_sphere: int = -1
    rot_axis_point: tuple = (0.0, 0.0, 0.0)

    def blob(self):
        """Flat float32 scene description (see module docstring)."""
        h = np.zeros(HEADER_LEN, np.float32)
        h[0] = len(self.spheres)
        h[1] = len(self.boxes)
        h[2] = 1.0 if self.has_room else 0.0
        h[3] = self.rot_sphere
        h[4:7] = self.room_min
        h[7:10] = self.room_max
        h[10:13] = self.sky
        h[13:17] = self.skylight
        h[17] = self.wall_emission
        h[18:36] = np.asarray(self.wall_albedo, np.float32).reshape(-1)
        h[36:39] = self.rot_axis_point
        return np.concatenate([h, self.spheres.reshape(-1), self.boxes.reshape(-1)]).astype(np.float32)

    def at_time(self, t):
        """The same scene with the rotating sphere turned by 2*pi*t about +y (a copy)."""
        s = Scene(**{k: getattr(self, k) for k in self.__dataclass_fields__})
        s.spheres = self.spheres.copy()
        if self.rot_sphere >= 0:
            c = s.spheres[self.rot_sphere, :3].astype(np.float64) - np.asarray(self.rot_axis_point)
            a = 2.0 * math.pi * float(t)
            ca, sa = math.cos(a), math.sin(a)
            rx = ca * c[0] + sa * c[2]
            rz = -sa * c[0] + ca * c[2]
            s.spheres[self.rot_sphere, :3] = np.asarray(self.rot_axis_point) + np.array([rx, c[1], rz])
        return s


def _sphere_row(c, r, albedo, emission=(0.0, 0.0, 0.0)):
    row = np.zeros(SPHERE_LEN, np.float32)
    row[0:3] = c
    row[3] = r
    row[4:7] = albedo
    row[7:10] = emission
    return row


def _box_row(lo, hi, albedo):
    row = np.zeros(BOX_LEN, np.float32)
    row[0:3] = lo
    row[3:6] = hi
    row[6:9] = albedo
    return row


def _clear_of_emitter_path(c, r):
    """True if a ball (c, r) keeps 5 cm clear of the emitter's orbit tube (radius 3 at y=3)."""
    ring = math.hypot(math.hypot(c[0], c[2]) - math.hypot(EMITTER_CENTRE[0], EMITTER_CENTRE[2]),
                      c[1] - EMITTER_CENTRE[1])
    return ring > r + EMITTER_RADIUS + 0.05


def room_scene(seed=0, n_spheres=24, n_boxes=8, sky=1.0, with_emitter=True):
    """The 10 m closed room with a 4 m x 4 m skylight, random spheres/boxes and one sphere emitter.

    Spheres: radius U(0.2, 1.5); boxes: half-extents U(0.2, 1.0); centres uniform
    with the object fully inside the room; albedo U(0.1, 0.9) per channel.
    Objects that contain the camera or touch the emitter's orbit are redrawn.
    The emitter (radius 0.5, radiance 20, black) is the last sphere and rotates
    about the vertical axis through the room centre with the time input.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(ROOM_MIN)
    hi = np.asarray(ROOM_MAX)
    cam = np.asarray(CAMERA_POS)
    spheres = []
    while len(spheres) < n_spheres:
        r = rng.uniform(0.2, 1.5)
        c = rng.uniform(lo + r, hi - r)
        if np.linalg.norm(c - cam) <= r + 0.05 or not _clear_of_emitter_path(c, r):
            continue
        spheres.append(_sphere_row(c, r, rng.uniform(0.1, 0.9, 3)))
    boxes = []
    while len(boxes) < n_boxes:
        he = rng.uniform(0.2, 1.0, 3)
        c = rng.uniform(lo + he, hi - he)
        if np.all(np.abs(cam - c) <= he + 0.05) or not _clear_of_emitter_path(c, float(np.linalg.norm(he))):
            continue
        boxes.append(_box_row(c - he, c + he, rng.uniform(0.1, 0.9, 3)))
    rot = -1
    if with_emitter:
        spheres.append(_sphere_row(EMITTER_CENTRE, EMITTER_RADIUS, (0.0, 0.0, 0.0),
                                   (EMITTER_RADIANCE,) * 3))
        rot = len(spheres) - 1
    return Scene(
        spheres=np.asarray(spheres, np.float32).reshape(-1, SPHERE_LEN),
        boxes=np.asarray(boxes, np.float32).reshape(-1, BOX_LEN),
        has_room=True, sky=(sky, sky, sky), skylight=SKYLIGHT, rot_sphere=rot,
    )


def empty_scene(sky=1.0):
    """No geometry at all: every ray escapes to a uniform sky of radiance ``sky``."""
    return Scene(sky=(sky, sky, sky))


def single_emitter_scene(centre, radius, radiance):
    """One emitting sphere in empty black space."""
    s = _sphere_row(centre, radius, (0.0, 0.0, 0.0), (radiance,) * 3)
    return Scene(spheres=s.reshape(1, SPHERE_LEN))


def furnace_scene(albedo, wall_emission):
    """Closed room whose six walls all emit ``wall_emission`` and reflect ``albedo``."""
    a = (albedo, albedo, albedo)
    return Scene(has_room=True, wall_emission=wall_emission, wall_albedo=(a,) * 6)
