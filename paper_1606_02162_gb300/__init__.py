"""GiLA k-hop Fruchterman-Reingold layout on GB300."""
