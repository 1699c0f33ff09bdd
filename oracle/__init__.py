"""FP64 CPU oracle of the map-maker (test infrastructure only; see ``oracle.mapmaker``)."""
