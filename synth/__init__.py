from . import geometry, helix, events, maps
